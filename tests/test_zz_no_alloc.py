"""The allocation-free entry point, abcore_compute_static.

It serves callers that cannot allocate device memory at run time (code inside a framework that
owns the device's memory pool, plugins that must not grow a process's device footprint): its
working memory is a fixed array inside the library. Its masks must equal those of the ordinary
entry point, abcore_compute, on two calls in a row -- the array keeps the previous call's
contents, so the second call shows that each call clears what must start empty.

This file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2606_07148_gb300 import ABCore, abi


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


@pytest.mark.gpu
def test_static_entry_matches_compute_on_two_calls_in_a_row():
    from paper_2606_07148_gb300.buildlib import build
    build()
    nU, nV, m = 300_000, 150_000, 3_000_000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.4, seed=31, device="cuda")
    off, adj = _unified_csr(nU, nV, eu.cpu().numpy(), ev.cpu().numpy())
    d_off = torch.from_numpy(off).cuda()
    d_adj = torch.from_numpy(adj).cuda()
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    stream = torch.cuda.current_stream()
    handle = ctypes.c_void_p(stream.cuda_stream or 1)
    for a, b in [(3, 5), (12, 8)]:
        mu = torch.full((nU,), 7, dtype=torch.uint8, device="cuda")
        mv = torch.full((nV,), 7, dtype=torch.uint8, device="cuda")
        rc = abi.abcore_compute_static(nU, nV, _ptr(d_off), _ptr(d_adj), a, b, _ptr(mu), _ptr(mv), handle)
        assert rc == abi.ABCORE_OK
        wu, wv = core.compute(a, b)
        torch.cuda.synchronize()
        assert torch.equal(mu, wu) and torch.equal(mv, wv), (a, b)
        assert 0 < int(wu.sum()) < nU
    core.close()
