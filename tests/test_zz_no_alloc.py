"""The allocation-free entry point, abcore_compute_static.

It serves callers that cannot allocate device memory at run time (code inside a framework that
owns the device's memory pool, plugins that must not grow a process's device footprint): its
working memory is a fixed array inside the library. Its masks must equal those of the ordinary
entry point, abcore_compute, on two calls in a row -- the array keeps the previous call's
contents, so the second call shows that each call clears what must start empty -- and those of
the CPU oracle, on the same calls and on the degenerate cases (zero bounds, isolated vertices, an
empty core). Inputs it must refuse are refused before anything touches memory they describe.

This file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth
from paper_2606_07148_gb300 import abi


def _unified_csr(nU, nV, eu, ev):
    """Rows 0..nU-1 list nU + v, rows nU.. list u; every edge in both rows (plain bookkeeping)."""
    src = np.concatenate([eu, ev + nU]).astype(np.int64)
    dst = np.concatenate([ev + nU, eu]).astype(np.int32)
    order = np.argsort(src, kind="stable")
    off = np.zeros(nU + nV + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=nU + nV), out=off[1:])
    return off, dst[order]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_entry_rejects_graphs_beyond_its_limit():
    abi.load_library()
    too_many = abi.ABCORE_STATIC_MAX_VERTICES
    rc = abi.abcore_compute_static(too_many, 1, None, None, 1, 1, None, None, None)
    assert rc == abi.ABCORE_EINVAL
    assert abi.abcore_compute_static(1, 1, None, None, -1, 1, None, None, None) == abi.ABCORE_EINVAL


def _static(torch, nU, nV, d_off, d_adj, a, b, handle):
    mu = torch.full((max(nU, 1),), 7, dtype=torch.uint8, device="cuda")
    mv = torch.full((max(nV, 1),), 7, dtype=torch.uint8, device="cuda")
    rc = abi.abcore_compute_static(nU, nV, _ptr(d_off), _ptr(d_adj), a, b, _ptr(mu), _ptr(mv), handle)
    return rc, mu[:nU].cpu().numpy(), mv[:nV].cpu().numpy()


@pytest.mark.gpu
def test_static_entry_matches_compute_and_oracle_on_two_calls_in_a_row():
    import torch
    from paper_2606_07148_gb300 import ABCore
    from paper_2606_07148_gb300.buildlib import build
    build()
    nU, nV, m = 300_000, 150_000, 3_000_000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.4, seed=31, device="cuda")
    eu_h, ev_h = eu.cpu().numpy(), ev.cpu().numpy()
    off, adj = _unified_csr(nU, nV, eu_h, ev_h)
    ooff, oadj = oracle.build_csr(nU, nV, eu_h, ev_h)
    d_off = torch.from_numpy(off).cuda()
    d_adj = torch.from_numpy(adj).cuda()
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    stream = torch.cuda.current_stream()
    handle = ctypes.c_void_p(stream.cuda_stream or 1)
    for a, b in [(3, 5), (12, 8)]:
        rc, mu, mv = _static(torch, nU, nV, d_off, d_adj, a, b, handle)
        assert rc == abi.ABCORE_OK
        wu, wv = core.compute(a, b)
        torch.cuda.synchronize()
        assert np.array_equal(mu, wu.cpu().numpy()) and np.array_equal(mv, wv.cpu().numpy()), (a, b)
        ou, ov = oracle.peel(nU, nV, ooff, oadj, a, b)
        assert np.array_equal(mu, ou) and np.array_equal(mv, ov), (a, b)
        assert 0 < int(ou.sum()) < nU
    # zero bounds and a core that is empty, against the oracle
    for a, b in [(0, 0), (0, 7), (9, 0), (5000, 5000)]:
        rc, mu, mv = _static(torch, nU, nV, d_off, d_adj, a, b, handle)
        assert rc == abi.ABCORE_OK
        ou, ov = oracle.peel(nU, nV, ooff, oadj, a, b)
        assert np.array_equal(mu, ou) and np.array_equal(mv, ov), (a, b)
    assert int(ou.sum()) + int(ov.sum()) == 0
    core.close()


@pytest.mark.gpu
def test_static_entry_isolated_vertices_and_refused_inputs():
    import torch
    from paper_2606_07148_gb300.buildlib import build
    build()
    handle = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream or 1)
    # a small graph whose last vertices of each layer are isolated: queued with no row to walk
    nU, nV = 40, 30
    rng = np.random.default_rng(5)
    keys = rng.choice(30 * 20, size=200, replace=False)
    eu, ev = (keys // 20).astype(np.int32), (keys % 20).astype(np.int32)
    off, adj = _unified_csr(nU, nV, eu, ev)
    ooff, oadj = oracle.build_csr(nU, nV, eu, ev)
    d_off = torch.from_numpy(off).cuda()
    d_adj = torch.from_numpy(adj).cuda()
    for a, b in [(0, 0), (1, 1), (3, 4), (0, 3), (2, 0), (50, 50)]:
        rc, mu, mv = _static(torch, nU, nV, d_off, d_adj, a, b, handle)
        assert rc == abi.ABCORE_OK
        ou, ov = oracle.peel(nU, nV, ooff, oadj, a, b)
        assert np.array_equal(mu, ou) and np.array_equal(mv, ov), (a, b)
    # rows needing one queue item more than the array holds: refused by the size check, which
    # reads the offsets only (the one-entry adj is never read)
    big = 1024 * (abi.ABCORE_STATIC_MAX_ITEMS + 1)
    d_big = torch.tensor([0, big, big], dtype=torch.int64, device="cuda")
    d_one = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc, _, _ = _static(torch, 1, 1, d_big, d_one, 1, 1, handle)
    assert rc == abi.ABCORE_EINVAL
    # exactly at the limit is accepted by the size check: ABCORE_STATIC_MAX_ITEMS rows of one
    # entry each would need too many vertices, so take one row of 1024 * (limit - 1) entries
    # plus one empty row -- refused only if the count were not exact (it is within the limit);
    # the peel of (0, 0) never walks a row, so the large row is not read
    ok_len = 1024 * (abi.ABCORE_STATIC_MAX_ITEMS - 1)
    d_ok = torch.tensor([0, ok_len, ok_len], dtype=torch.int64, device="cuda")
    rc, mu, mv = _static(torch, 1, 1, d_ok, d_one, 0, 0, handle)
    assert rc == abi.ABCORE_OK and mu.tolist() == [1] and mv.tolist() == [1]
    # decreasing offsets
    d_dec = torch.tensor([0, 5, 3], dtype=torch.int64, device="cuda")
    rc, _, _ = _static(torch, 1, 1, d_dec, d_one, 1, 1, handle)
    assert rc == abi.ABCORE_EINVAL
    # an adjacency id that is not a vertex: found where the cascade reads it, never used
    d_off2 = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda")
    d_bad = torch.tensor([7, 0], dtype=torch.int32, device="cuda")
    rc, _, _ = _static(torch, 1, 1, d_off2, d_bad, 5, 5, handle)
    assert rc == abi.ABCORE_EINVAL
    # and the array is usable again afterwards
    rc, mu, mv = _static(torch, nU, nV, d_off, d_adj, 3, 4, handle)
    ou, ov = oracle.peel(nU, nV, ooff, oadj, 3, 4)
    assert rc == abi.ABCORE_OK and np.array_equal(mu, ou) and np.array_equal(mv, ov)
