"""ctypes binding of the C ABI in include/abcore.h, with the same function names.

Argument marshalling only: every computation happens in libabcore.so's CUDA kernels. Loading
fails loudly if the library has not been built -- there is no fallback path.
"""

import ctypes
import os

from .buildlib import LIB

ABCORE_OK = 0
ABCORE_EINVAL = -1
ABCORE_ENOTLOADED = -2
ABCORE_ENOMEM = -3
ABCORE_EEXIST = -4
ABCORE_ENOENT = -5
ABCORE_ECUDA = -6
ABCORE_ETIMEDOUT = -7
ABCORE_EBUSY = -8

ABCORE_TUNE_PEEL = 0
ABCORE_TUNE_BATCH = 1
ABCORE_PTR_HOST = 0
ABCORE_PTR_DEVICE = 1
ABCORE_VALIDATE = 2
ABCORE_ASYNC = 4

ABCORE_INSERT = 0
ABCORE_DELETE = 1

EXPORTED = [
    "abcore_create", "abcore_destroy", "abcore_last_error", "abcore_load_edges", "abcore_load_csr",
    "abcore_compute", "abcore_compute_batch", "abcore_sync", "abcore_components", "abcore_core_numbers", "abcore_autotune",
    "abcore_alpha_offset", "abcore_default_query", "abcore_community", "abcore_measure_atomics", "abcore_query_edge",
    "abcore_serve_start", "abcore_serve_submit", "abcore_serve_poll", "abcore_serve_stop",
    "abcore_get_stats", "abcore_set_param", "abcore_get_param", "abcore_graph_info", "abcore_export_csr",
    "abcore_compute_static",
]

ABCORE_STATIC_MAX_VERTICES = 1 << 20
ABCORE_STATIC_MAX_ITEMS = (1 << 20) + (1 << 16)


K_INIT, K_STREAM, K_CASCADE, K_BATCH, K_SERVE = 0, 1, 2, 3, 4
K_KINDS = 8


class abcore_stats(ctypes.Structure):
    _fields_ = [
        ("peels", ctypes.c_int64), ("candidates", ctypes.c_int64), ("init_vertices", ctypes.c_int64),
        ("search_probes", ctypes.c_int64), ("stream_entries", ctypes.c_int64), ("entries", ctypes.c_int64),
        ("decrements", ctypes.c_int64), ("stream_decrements", ctypes.c_int64), ("scanned", ctypes.c_int64), ("pushes", ctypes.c_int64),
        ("items", ctypes.c_int64),
        ("emit_gathered", ctypes.c_int64), ("emit_scattered", ctypes.c_int64), ("mask_zeroed", ctypes.c_int64),
        ("launches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64 * K_KINDS),
        ("kernel_ms", ctypes.c_double * K_KINDS), ("mode", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
        ("device_bytes", ctypes.c_int64), ("peak_device_bytes", ctypes.c_int64),
        ("round0_rows", ctypes.c_int64), ("scope_queries", ctypes.c_int64), ("scope_vertices", ctypes.c_int64),
        ("serve_regions", ctypes.c_int64), ("serve_region_vertices", ctypes.c_int64),
        ("serve_cascades", ctypes.c_int64), ("serve_cascade_vertices", ctypes.c_int64),
        ("hub_decrements", ctypes.c_int64), ("hub_flushes", ctypes.c_int64),
    ]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        return d


class abcore_req(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("u", ctypes.c_int32), ("v", ctypes.c_int32),
                ("target", ctypes.c_int32), ("tag", ctypes.c_uint64)]


class abcore_resp(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("in_core", ctypes.c_uint8), ("u_in", ctypes.c_uint8), ("v_in", ctypes.c_uint8),
                ("pad", ctypes.c_uint8)]


_lib = None
_vp = ctypes.c_void_p


def load_library(path: str = LIB):
    """Load libabcore.so; raises if it is missing (build it with paper_2606_07148_gb300.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libabcore.so is not built (%s); run paper_2606_07148_gb300.build()" % path)
    lib = ctypes.CDLL(path)
    sig = {
        "abcore_create": ([ctypes.POINTER(_vp), ctypes.c_int, _vp], ctypes.c_int),
        "abcore_destroy": ([_vp], ctypes.c_int),
        "abcore_last_error": ([_vp], ctypes.c_char_p),
        "abcore_load_edges": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _vp, _vp, ctypes.c_uint32],
                              ctypes.c_int),
        "abcore_load_csr": ([_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_uint32], ctypes.c_int),
        "abcore_compute": ([_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, ctypes.c_uint32], ctypes.c_int),
        "abcore_compute_batch": ([_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_uint32], ctypes.c_int),
        "abcore_sync": ([_vp], ctypes.c_int),
        "abcore_autotune": ([_vp, ctypes.c_int32, _vp, _vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)],
                            ctypes.c_int),
        "abcore_alpha_offset": ([_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "abcore_default_query": ([_vp] + [ctypes.POINTER(ctypes.c_int32)] * 4, ctypes.c_int),
        "abcore_community": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                              ctypes.POINTER(ctypes.c_int64), ctypes.c_uint32], ctypes.c_int),
        "abcore_measure_atomics": ([_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "abcore_core_numbers": ([_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_uint32], ctypes.c_int),
        "abcore_components": ([_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_uint32], ctypes.c_int),
        "abcore_query_edge": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_uint8)], ctypes.c_int),
        "abcore_serve_start": ([_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
        "abcore_serve_submit": ([_vp, _vp, ctypes.c_int32, _vp], ctypes.c_int),
        "abcore_serve_poll": ([_vp, _vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "abcore_serve_stop": ([_vp], ctypes.c_int),
        "abcore_get_stats": ([_vp, ctypes.POINTER(abcore_stats)], ctypes.c_int),
        "abcore_set_param": ([_vp, ctypes.c_char_p, ctypes.c_int64], ctypes.c_int),
        "abcore_get_param": ([_vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "abcore_graph_info": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "abcore_export_csr": ([_vp, _vp, _vp, _vp, ctypes.c_uint32], ctypes.c_int),
        "abcore_compute_static": ([ctypes.c_int32, ctypes.c_int32, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                   _vp, _vp, _vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _fn(name):
    def call(*args):
        return getattr(load_library(), name)(*args)
    call.__name__ = name
    return call


abcore_create = _fn("abcore_create")
abcore_destroy = _fn("abcore_destroy")
abcore_last_error = _fn("abcore_last_error")
abcore_load_edges = _fn("abcore_load_edges")
abcore_load_csr = _fn("abcore_load_csr")
abcore_compute = _fn("abcore_compute")
abcore_compute_batch = _fn("abcore_compute_batch")
abcore_sync = _fn("abcore_sync")
abcore_components = _fn("abcore_components")
abcore_core_numbers = _fn("abcore_core_numbers")
abcore_autotune = _fn("abcore_autotune")
abcore_alpha_offset = _fn("abcore_alpha_offset")
abcore_default_query = _fn("abcore_default_query")
abcore_community = _fn("abcore_community")
abcore_measure_atomics = _fn("abcore_measure_atomics")
abcore_query_edge = _fn("abcore_query_edge")
abcore_serve_start = _fn("abcore_serve_start")
abcore_serve_submit = _fn("abcore_serve_submit")
abcore_serve_poll = _fn("abcore_serve_poll")
abcore_serve_stop = _fn("abcore_serve_stop")
abcore_get_stats = _fn("abcore_get_stats")
abcore_set_param = _fn("abcore_set_param")
abcore_get_param = _fn("abcore_get_param")
abcore_graph_info = _fn("abcore_graph_info")
abcore_export_csr = _fn("abcore_export_csr")
abcore_compute_static = _fn("abcore_compute_static")
