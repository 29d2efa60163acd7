"""Input generators: determinism, exact edge counts, valid update streams, grid values."""

import numpy as np
import torch

import synth


def test_chung_lu_exact_distinct_and_deterministic():
    for (nU, nV, m, gu, gv, seed) in [(2000, 1500, 20000, 2.3, 2.3, 0), (300, 50, 4000, 2.1, 2.4, 1),
                                      (10, 10, 100, 2.0, 2.0, 2)]:
        eu, ev = synth.chung_lu_edges(nU, nV, m, gu, gv, seed)
        eu2, ev2 = synth.chung_lu_edges(nU, nV, m, gu, gv, seed)
        assert torch.equal(eu, eu2) and torch.equal(ev, ev2)
        assert eu.dtype == torch.int32 and eu.numel() == m
        assert int(eu.min()) >= 0 and int(eu.max()) < nU and int(ev.min()) >= 0 and int(ev.max()) < nV
        assert (eu.long() * nV + ev.long()).unique().numel() == m


def test_chung_lu_buckets_give_same_law():
    """Splitting the draw into several U buckets still yields m distinct in-range edges."""
    eu, ev = synth.chung_lu_edges(5000, 3000, 60000, 2.1, 2.2, 5, bucket_edges=8000)
    assert eu.numel() == 60000 and (eu.long() * 3000 + ev.long()).unique().numel() == 60000


def test_power_law_weights():
    w = synth.layer_weights(100000, 2.1, 2_000_000)
    assert abs(w.sum() - 2_000_000) < 1e-3 * 2_000_000
    assert w.max() <= int(np.sqrt(2_000_000)) and w.min() >= 1.0
    assert np.all(np.diff(w) <= 1e-9)


def test_grids():
    assert synth.log_grid(16, 1, 512) == [1, 2, 3, 4, 5, 8, 12, 18, 28, 42, 64, 97, 147, 223, 338, 512]
    assert synth.log_grid(8, 1, 1024) == [1, 3, 7, 20, 53, 141, 380, 1024]
    assert len(synth.grid_pairs(16, 1, 512)) == 256


def test_update_stream_is_valid_sequence():
    nU, nV = 300, 200
    eu, ev = synth.chung_lu_edges(nU, nV, 3000, 2.1, 2.2, 4)
    s = synth.edge_update_stream(eu.numpy(), ev.numpy(), nU, nV, 3000, 4)
    cur = set(zip(eu.tolist(), ev.tolist()))
    for k in range(len(s)):
        e = (int(s.u[k]), int(s.v[k]))
        if s.op[k] == 0:
            assert e not in cur
            cur.add(e)
        else:
            assert e in cur
            cur.discard(e)
    frac = float((s.op == 0).mean())
    assert 0.6 < frac < 0.8
    assert set(np.unique(s.target).tolist()) <= {0, 1, 2, 3}
    assert np.all(np.diff(s.t_unit) > 0)
    s2 = synth.edge_update_stream(eu.numpy(), ev.numpy(), nU, nV, 3000, 4)
    assert np.array_equal(s.u, s2.u) and np.array_equal(s.op, s2.op)
