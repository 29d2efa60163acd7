"""Exact (alpha, beta)-core computation on bipartite graphs for one GB300 (sm_103a).

``abi`` is the ctypes binding of include/abcore.h (same names). ``ABCore`` is a thin
convenience wrapper that marshals torch tensors and numpy arrays into those calls; PyTorch
provides device memory and streams only, every step runs in the library's CUDA kernels.
"""

import ctypes

import numpy as np

from . import abi
from .buildlib import build, LIB

__all__ = ["abi", "build", "LIB", "ABCore", "ABCoreError"]


class ABCoreError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("abcore error %d: %s" % (code, msg))
        self.code = code


def _torch():
    import torch
    return torch


class ABCore:
    """One library context on one CUDA device, ordered on one stream."""

    def __init__(self, device: int = 0, stream=None):
        """Work is ordered on ``stream`` (default: torch's current stream on ``device``), so
        tensors produced by torch on that stream are complete before the library reads them."""
        abi.load_library()
        torch = _torch()
        self._h = ctypes.c_void_p()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        # torch reports its legacy default stream as handle 0; the C ABI reads NULL as "create a
        # private stream", so pass cudaStreamLegacy (handle 1) for it instead.
        self.stream = stream
        s = ctypes.c_void_p(stream.cuda_stream or 1)
        rc = abi.abcore_create(ctypes.byref(self._h), device, s)
        if rc != 0:
            raise ABCoreError(rc, "abcore_create failed")
        self.device = device
        self.nU = self.nV = self.m = 0

    # -- helpers ---------------------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise ABCoreError(rc, abi.abcore_last_error(self._h).decode(errors="replace"))
        return rc

    def close(self):
        if self._h:
            abi.abcore_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _ptr(x):
        """(pointer, flags) of a contiguous torch tensor or numpy array."""
        torch = _torch()
        if isinstance(x, torch.Tensor):
            assert x.is_contiguous()
            return ctypes.c_void_p(x.data_ptr()), (abi.ABCORE_PTR_DEVICE if x.is_cuda else abi.ABCORE_PTR_HOST)
        a = np.ascontiguousarray(x)
        return ctypes.c_void_p(a.ctypes.data), abi.ABCORE_PTR_HOST

    # -- loading ---------------------------------------------------------------------------
    def load_edges(self, nU, nV, eu, ev):
        torch = _torch()
        if isinstance(eu, torch.Tensor):
            eu = eu.to(torch.int32).contiguous()
            ev = ev.to(torch.int32).contiguous()
            assert eu.is_cuda == ev.is_cuda
        else:
            eu = np.ascontiguousarray(eu, dtype=np.int32)
            ev = np.ascontiguousarray(ev, dtype=np.int32)
        pu, fl = self._ptr(eu)
        pv, _ = self._ptr(ev)
        m = int(eu.numel() if isinstance(eu, torch.Tensor) else eu.size)
        self._check(abi.abcore_load_edges(self._h, nU, nV, m, pu, pv, fl))
        self.nU, self.nV, self.m = nU, nV, m

    def load_csr(self, nU, nV, offU, adjU, offV=None, adjV=None, validate=False):
        offU = np.ascontiguousarray(offU, dtype=np.int64)
        adjU = np.ascontiguousarray(adjU, dtype=np.int32)
        args = [self._ptr(offU)[0], self._ptr(adjU)[0]]
        if offV is not None:
            offV = np.ascontiguousarray(offV, dtype=np.int64)
            adjV = np.ascontiguousarray(adjV, dtype=np.int32)
            args += [self._ptr(offV)[0], self._ptr(adjV)[0]]
        else:
            args += [None, None]
        fl = abi.ABCORE_PTR_HOST | (abi.ABCORE_VALIDATE if validate else 0)
        self._check(abi.abcore_load_csr(self._h, nU, nV, *args, fl))
        self.nU, self.nV, self.m = nU, nV, int(offU[nU])

    # -- computation -----------------------------------------------------------------------
    def compute(self, alpha, beta, out_u=None, out_v=None, asynchronous=False):
        """Masks (uint8 0/1) of the (alpha, beta)-core; device tensors unless outputs are given."""
        torch = _torch()
        if out_u is None:
            out_u = torch.empty(self.nU, dtype=torch.uint8, device="cuda:%d" % self.device)
            out_v = torch.empty(self.nV, dtype=torch.uint8, device="cuda:%d" % self.device)
        pu, fl = self._ptr(out_u)
        pv, _ = self._ptr(out_v)
        if asynchronous:
            fl |= abi.ABCORE_ASYNC
        self._check(abi.abcore_compute(self._h, int(alpha), int(beta), pu, pv, fl))
        return out_u, out_v

    def compute_batch(self, alphas, betas, out_u=None, out_v=None, asynchronous=False):
        torch = _torch()
        n = len(alphas)
        a = np.ascontiguousarray(alphas, dtype=np.int32)
        b = np.ascontiguousarray(betas, dtype=np.int32)
        if out_u is None:
            out_u = torch.empty((n, self.nU), dtype=torch.uint8, device="cuda:%d" % self.device)
            out_v = torch.empty((n, self.nV), dtype=torch.uint8, device="cuda:%d" % self.device)
        pu, fl = self._ptr(out_u)
        pv, _ = self._ptr(out_v)
        if asynchronous:
            fl |= abi.ABCORE_ASYNC
        self._check(abi.abcore_compute_batch(self._h, n, a.ctypes.data_as(ctypes.c_void_p),
                                             b.ctypes.data_as(ctypes.c_void_p), pu, pv, fl))
        return out_u, out_v

    def autotune(self, pairs, batch=False):
        """Tune the launch parameters on a sample of (alpha, beta) pairs; returns the best sample
        time in ms and the chosen parameters."""
        a = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
        b = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
        best = ctypes.c_double(0)
        what = abi.ABCORE_TUNE_BATCH if batch else abi.ABCORE_TUNE_PEEL
        self._check(abi.abcore_autotune(self._h, len(pairs), a.ctypes.data_as(ctypes.c_void_p),
                                        b.ctypes.data_as(ctypes.c_void_p), what, ctypes.byref(best)))
        return best.value, {k: self.get_param(k) for k in self.TUNED}

    def measure_atomics(self, array_bytes=32 << 20):
        """Random 32-bit atomicSub throughput (per second), with and without the returned value."""
        w, wo = ctypes.c_double(0), ctypes.c_double(0)
        self._check(abi.abcore_measure_atomics(self._h, int(array_bytes), ctypes.byref(w), ctypes.byref(wo)))
        return w.value, wo.value

    def sync(self):
        self._check(abi.abcore_sync(self._h))

    def core_numbers(self, out_u=None, out_v=None):
        """Core numbers (int32, Definition 2) and the largest; prepares the GCC+ pruned peel."""
        torch = _torch()
        if out_u is None:
            out_u = torch.empty(self.nU, dtype=torch.int32, device="cuda:%d" % self.device)
            out_v = torch.empty(self.nV, dtype=torch.int32, device="cuda:%d" % self.device)
        pu, fl = self._ptr(out_u)
        pv, _ = self._ptr(out_v)
        mx = ctypes.c_int32(0)
        self._check(abi.abcore_core_numbers(self._h, pu, pv, ctypes.byref(mx), fl))
        return out_u, out_v, int(mx.value)

    def alpha_offset(self, alpha):
        """Largest beta >= 1 with a non-empty (alpha, beta)-core (0 if none)."""
        b = ctypes.c_int32(0)
        self._check(abi.abcore_alpha_offset(self._h, int(alpha), ctypes.byref(b)))
        return int(b.value)

    def default_query(self):
        """The paper's default query (Section 6), computed by the library: returns
        (delta, alpha, alpha_offset, beta)."""
        out = [ctypes.c_int32(0) for _ in range(4)]
        self._check(abi.abcore_default_query(self._h, *[ctypes.byref(x) for x in out]))
        return tuple(int(x.value) for x in out)

    def community(self, layer, vid, alpha, beta, out_u=None, out_v=None):
        """Masks of the (alpha, beta)-core's component containing vertex vid of layer (0 U, 1 V)."""
        torch = _torch()
        if out_u is None:
            out_u = torch.empty(self.nU, dtype=torch.uint8, device="cuda:%d" % self.device)
            out_v = torch.empty(self.nV, dtype=torch.uint8, device="cuda:%d" % self.device)
        pu, fl = self._ptr(out_u)
        pv, _ = self._ptr(out_v)
        size = ctypes.c_int64(0)
        self._check(abi.abcore_community(self._h, int(layer), int(vid), int(alpha), int(beta), pu, pv,
                                         ctypes.byref(size), fl))
        return out_u, out_v, int(size.value)

    def components(self, out_u=None, out_v=None):
        """Component labels (int32, the smallest unified caller id in each component) and the
        number of components; device tensors unless outputs are given."""
        torch = _torch()
        if out_u is None:
            out_u = torch.empty(self.nU, dtype=torch.int32, device="cuda:%d" % self.device)
            out_v = torch.empty(self.nV, dtype=torch.int32, device="cuda:%d" % self.device)
        pu, fl = self._ptr(out_u)
        pv, _ = self._ptr(out_v)
        nc = ctypes.c_int64(0)
        self._check(abi.abcore_components(self._h, pu, pv, ctypes.byref(nc), fl))
        return out_u, out_v, int(nc.value)

    def query_edge(self, u, v, op, alpha, beta):
        r = ctypes.c_uint8(0)
        self._check(abi.abcore_query_edge(self._h, int(u), int(v), int(op), int(alpha), int(beta), ctypes.byref(r)))
        return int(r.value)

    # -- serving ---------------------------------------------------------------------------
    def serve_start(self, targets, ring_slots=4096):
        a = np.ascontiguousarray([t[0] for t in targets], dtype=np.int32)
        b = np.ascontiguousarray([t[1] for t in targets], dtype=np.int32)
        self._check(abi.abcore_serve_start(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                           b.ctypes.data_as(ctypes.c_void_p), len(targets), ring_slots))

    def serve_submit(self, reqs):
        """reqs: ctypes array of abi.abcore_req. Returns the sequence numbers, or None if busy."""
        n = len(reqs)
        seq = (ctypes.c_uint64 * max(n, 1))()
        rc = abi.abcore_serve_submit(self._h, ctypes.cast(reqs, ctypes.c_void_p), n, ctypes.cast(seq, ctypes.c_void_p))
        if rc == abi.ABCORE_EBUSY:
            return None
        self._check(rc)
        return list(seq[:n])

    def serve_poll(self, max_n=4096):
        out = (abi.abcore_resp * max_n)()
        got = ctypes.c_int32(0)
        self._check(abi.abcore_serve_poll(self._h, ctypes.cast(out, ctypes.c_void_p), max_n, ctypes.byref(got)))
        return out[:got.value]

    RESP_DTYPE = np.dtype([("seq", "<u8"), ("tag", "<u8"), ("status", "<i4"), ("in_core", "u1"),
                           ("u_in", "u1"), ("v_in", "u1"), ("pad", "u1")])

    def serve_poll_into(self, buf):
        """Poll into a reusable numpy array of RESP_DTYPE; returns the filled prefix (a view).
        Creates no Python object per response, so a long stream leaves nothing for the
        garbage collector to walk."""
        got = ctypes.c_int32(0)
        self._check(abi.abcore_serve_poll(self._h, ctypes.c_void_p(buf.ctypes.data), len(buf), ctypes.byref(got)))
        return buf[:got.value]

    def serve_stop(self):
        self._check(abi.abcore_serve_stop(self._h))

    # -- introspection ---------------------------------------------------------------------
    def stats(self):
        s = abi.abcore_stats()
        self._check(abi.abcore_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def set_param(self, name, value):
        self._check(abi.abcore_set_param(self._h, name.encode(), int(value)))

    def get_param(self, name):
        v = ctypes.c_int64(0)
        self._check(abi.abcore_get_param(self._h, name.encode(), ctypes.byref(v)))
        return int(v.value)

    TUNED = ("blocks_per_sm", "chunk", "grab_div", "batch_entries", "flush_steps", "hub_degree", "probe_bytes",
             "emit_scatter_max_pct", "emit_bitmap_min_pct", "round0", "round0_variant", "round0_hub", "batch_entries_small",
             "batch_wave", "batch_seed", "batch_plain_below")

    def graph_info(self):
        nU, nV, du, dv = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        m = ctypes.c_int64()
        self._check(abi.abcore_graph_info(self._h, ctypes.byref(nU), ctypes.byref(nV), ctypes.byref(m),
                                          ctypes.byref(du), ctypes.byref(dv)))
        return dict(nU=nU.value, nV=nV.value, m=m.value, max_deg_u=du.value, max_deg_v=dv.value)

    def export_csr(self):
        n = self.nU + self.nV
        off = np.zeros(n + 1, dtype=np.int64)
        adj = np.zeros(max(2 * self.m, 1), dtype=np.int32)
        n2o = np.zeros(max(n, 1), dtype=np.int32)
        self._check(abi.abcore_export_csr(self._h, off.ctypes.data_as(ctypes.c_void_p),
                                          adj.ctypes.data_as(ctypes.c_void_p),
                                          n2o.ctypes.data_as(ctypes.c_void_p), abi.ABCORE_PTR_HOST))
        return off, adj[: 2 * self.m], n2o[:n]
