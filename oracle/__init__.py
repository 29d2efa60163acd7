"""CPU oracle for exact (alpha, beta)-cores -- TEST INFRASTRUCTURE.

Plain, slow, single-threaded C (``abcore_oracle.c``) behind ctypes. Only the tests, the smoke
check and the benchmark's CPU-baseline leg use it; the CUDA library never imports or calls it,
and the two share no code. Vertex ids are unified: U vertex u is u, V vertex v is nU + v.

Parity status of each function (what pins it, see ``tests/test_oracle_pins.py``):

* ``build_csr``     -- pinned: per-row neighbour sets against a direct Python construction.
* ``peel``          -- pinned: brute-force subset enumeration on every graph with |U|, |V| <= 3
  and on random graphs of <= 14 vertices; closed forms ((0,0), (1,beta), (alpha,1), complete
  bipartite, forests, even cycles); the (k,k)-core against networkx's k-core; Lemma 1; the
  nested property; the paper's worked examples.
* ``core_numbers``  -- pinned against networkx.core_number.
* ``replay``        -- pinned: brute force on tiny update streams.
* ``components``    -- pinned: scipy.sparse.csgraph.connected_components on random graphs,
  closed forms (no edges, complete bipartite, perfect matchings, paths).
* ``default_query`` -- pinned: closed form on complete bipartite graphs (delta = min(a, b) and
  alpha_offset = |U|), and brute force of alpha_offset over every beta on random graphs.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abcore_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = "gcc -O2 -std=c11 -Wall -shared -fPIC -o %s %s" % (tmp, _SRC)
        if os.system(cmd) != 0:
            raise RuntimeError("oracle build failed: " + cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_build_csr.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                      _i32p, _i32p, _i64p, _i32p]
        lib.orc_peel_csr.argtypes = [ctypes.c_int32, ctypes.c_int32, _i64p, _i32p,
                                     ctypes.c_int32, ctypes.c_int32, _u8p]
        lib.orc_core_numbers.argtypes = [ctypes.c_int32, ctypes.c_int32, _i64p, _i32p, _i32p]
        lib.orc_components.argtypes = [ctypes.c_int32, ctypes.c_int32, _i64p, _i32p, _i32p,
                                       ctypes.POINTER(ctypes.c_int64)]
        lib.orc_components.restype = ctypes.c_int
        lib.orc_replay.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _i32p, _i32p,
                                   ctypes.c_int64, _i8p, _i32p, _i32p, _i32p, _i32p, _u8p,
                                   _i8p, _u8p, _i32p]
        for f in (lib.orc_build_csr, lib.orc_peel_csr, lib.orc_core_numbers, lib.orc_replay):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with code %d" % (what, code))
        self.code = code


def build_csr(nU, nV, eu, ev):
    """Unified CSR: off int64[nU+nV+1], adj int32[2m] (unified ids), rows sorted ascending."""
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    m = len(eu)
    off = np.zeros(nU + nV + 1, dtype=np.int64)
    adj = np.zeros(max(2 * m, 1), dtype=np.int32)
    rc = _load().orc_build_csr(nU, nV, m, eu, ev, off, adj)
    if rc != 0:
        raise OracleError(rc, "build_csr")
    return off, adj[: 2 * m]


def peel(nU, nV, off, adj, alpha, beta):
    """(mask_u, mask_v): uint8 0/1 membership of the (alpha, beta)-core."""
    alive = np.zeros(max(nU + nV, 1), dtype=np.uint8)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    rc = _load().orc_peel_csr(nU, nV, np.ascontiguousarray(off, dtype=np.int64), adj,
                              int(alpha), int(beta), alive)
    if rc != 0:
        raise OracleError(rc, "peel")
    return alive[:nU].copy(), alive[nU:nU + nV].copy()


def core_numbers(nU, nV, off, adj):
    """Core number (Definition 2) of every unified vertex."""
    core = np.zeros(max(nU + nV, 1), dtype=np.int32)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    rc = _load().orc_core_numbers(nU, nV, np.ascontiguousarray(off, dtype=np.int64), adj, core)
    if rc != 0:
        raise OracleError(rc, "core_numbers")
    return core[: nU + nV]


def replay(nU, nV, eu, ev, op, qu, qv, alpha, beta, check=None):
    """Apply the update stream in order; at checked steps, peel the updated graph from scratch.

    Returns (answer int8 [-1 = not checked, else 0/1], bits uint8, status int32) per op.
    """
    nops = len(op)
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    if len(eu) == 0:
        eu = np.zeros(1, dtype=np.int32)
        ev = np.zeros(1, dtype=np.int32)
        m = 0
    else:
        m = len(eu)
    if check is None:
        check = np.ones(nops, dtype=np.uint8)
    answer = np.zeros(max(nops, 1), dtype=np.int8)
    bits = np.zeros(max(nops, 1), dtype=np.uint8)
    status = np.zeros(max(nops, 1), dtype=np.int32)

    def arr(x, dt):
        a = np.ascontiguousarray(x, dtype=dt)
        return a if a.size else np.zeros(1, dtype=dt)

    rc = _load().orc_replay(nU, nV, m, eu, ev, nops, arr(op, np.int8), arr(qu, np.int32),
                            arr(qv, np.int32), arr(alpha, np.int32), arr(beta, np.int32),
                            arr(check, np.uint8), answer, bits, status)
    if rc != 0:
        raise OracleError(rc, "replay")
    return answer[:nops], bits[:nops], status[:nops]


def components(nU, nV, off, adj):
    """(labels int32[nU+nV], count): each vertex's component labelled by its smallest unified id."""
    label = np.zeros(max(nU + nV, 1), dtype=np.int32)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)
    nc = ctypes.c_int64(0)
    rc = _load().orc_components(nU, nV, np.ascontiguousarray(off, dtype=np.int64), adj, label, ctypes.byref(nc))
    if rc != 0:
        raise OracleError(rc, "components")
    return label[: nU + nV], int(nc.value)


def default_query(nU, nV, off, adj):
    """The paper's default query (Section 6), from its definition: delta is the largest core
    number; alpha = floor(0.4 delta), at least 1; alpha_offset is the largest beta >= 1 whose
    (alpha, beta)-core is non-empty (0 if none), found by trying beta = 1, 2, ... in turn until the
    core empties (the nested property makes every larger beta empty too); beta =
    floor(0.6 alpha_offset). The products are taken in integers. Returns
    (delta, alpha, alpha_offset, beta)."""
    core = core_numbers(nU, nV, off, adj)
    delta = int(core.max()) if core.size else 0
    alpha = max(1, (2 * delta) // 5)
    off_beta = 0
    if nU + nV > 0:
        beta = 1
        while True:
            mu, mv = peel(nU, nV, off, adj, alpha, beta)
            if int(mu.sum()) + int(mv.sum()) == 0:
                break
            off_beta = beta
            beta += 1
    return delta, alpha, off_beta, (3 * off_beta) // 5


# ------------------------------------------------------------------------------------------
# Many independent oracle runs side by side. Each run is the plain single-threaded oracle above;
# host threads only run several of them at once (ctypes releases the GIL during a call), so the
# checks of a large workload finish in minutes. Nothing is shared between runs but the inputs.
# ------------------------------------------------------------------------------------------
def default_threads():
    return max(1, min(8, (os.cpu_count() or 2) // 2))


def peel_many(nU, nV, off, adj, pairs, threads=None):
    """{(alpha, beta): (mask_u, mask_v, seconds)} for every distinct pair."""
    import concurrent.futures as cf
    import time

    def one(p):
        t = time.perf_counter()
        mu, mv = peel(nU, nV, off, adj, p[0], p[1])
        return p, (mu, mv, time.perf_counter() - t)

    with cf.ThreadPoolExecutor(max_workers=threads or default_threads()) as ex:
        return dict(ex.map(one, list(dict.fromkeys(tuple(p) for p in pairs))))


def replay_at(nU, nV, eu, ev, op, qu, qv, alpha, beta, ks, threads=None):
    """{k: (answer, bits, status)} of replay() at the update positions ks. The positions are split
    into groups of consecutive ones; each group is one replay of the stream up to its last
    position, checking only the group's positions."""
    import concurrent.futures as cf
    ks = sorted(set(int(k) for k in ks))
    if not ks:
        return {}
    t = max(1, min(threads or default_threads(), len(ks)))
    groups = [ks[i::t] for i in range(t)]

    def one(g):
        hi = g[-1] + 1
        check = np.zeros(hi, dtype=np.uint8)
        check[g] = 1
        ans, bits, st = replay(nU, nV, eu, ev, op[:hi], qu[:hi], qv[:hi], alpha[:hi], beta[:hi], check)
        return {k: (int(ans[k]), int(bits[k]), int(st[k])) for k in g}

    out = {}
    with cf.ThreadPoolExecutor(max_workers=t) as ex:
        for d in ex.map(one, groups):
            out.update(d)
    return out
