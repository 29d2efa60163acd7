"""GPU parity of the core decomposition (Definition 2) and of the pruned single query
(Lemma 1, Algorithm 2: GCC+) against the oracle's bucket-algorithm core numbers and its peel."""

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2606_07148_gb300 import ABCore, abi
from tests.bruteforce import load_paper_examples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_07148_gb300.buildlib import build
    build()


def _load(nU, nV, eu, ev):
    core = ABCore(0)
    core.load_edges(nU, nV, np.asarray(eu, np.int32), np.asarray(ev, np.int32))
    off, adj = oracle.build_csr(nU, nV, np.asarray(eu, np.int32), np.asarray(ev, np.int32))
    return core, off, adj


def _check_core_numbers(core, nU, nV, off, adj, host=False):
    want = oracle.core_numbers(nU, nV, off, adj)
    if host:
        cu, cv = np.zeros(nU, np.int32), np.zeros(nV, np.int32)
        _, _, mx = core.core_numbers(cu, cv)
    else:
        tu, tv, mx = core.core_numbers()
        cu, cv = tu.cpu().numpy(), tv.cpu().numpy()
    assert np.array_equal(cu, want[:nU]) and np.array_equal(cv, want[nU:])
    assert mx == (int(want.max()) if want.size else 0)
    return int(want.max()) if want.size else 0


def _check_pairs(core, nU, nV, off, adj, pairs):
    for a, b in pairs:
        mu, mv = core.compute(a, b)
        wu, wv = oracle.peel(nU, nV, off, adj, a, b)
        assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), (a, b)


def _pairs(kmax):
    vals = sorted({0, 1, 2, 3, 5, max(1, kmax // 2), kmax, kmax + 1, kmax + 7})
    return [(a, b) for a in vals for b in vals]


def test_core_numbers_and_pruned_peel_small_chung_lu():
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    core, off, adj = _load(nU, nV, eu.numpy(), ev.numpy())
    kmax = _check_core_numbers(core, nU, nV, off, adj)
    _check_core_numbers(core, nU, nV, off, adj, host=True)
    _check_pairs(core, nU, nV, off, adj, _pairs(kmax))
    st = core.stats()
    assert st["peels"] > 0
    core.close()


def test_pruned_and_plain_agree_on_the_serving_graph():
    nU, nV, eu, ev = synth.make_graph("serve-10kx5k-200k")
    core, off, adj = _load(nU, nV, eu.numpy(), ev.numpy())
    kmax = _check_core_numbers(core, nU, nV, off, adj)
    pairs = _pairs(kmax) + [(2, 2), (5, 5), (10, 20), (32, 32), (20, 10), (7, 40)]
    _check_pairs(core, nU, nV, off, adj, pairs)
    core.set_param("algo", 1)  # the plain peel on the same context
    _check_pairs(core, nU, nV, off, adj, [(10, 20), (3, 9)])
    core.close()


def test_paper_example_core_numbers():
    (nU, nV), edges, _ = load_paper_examples()
    core, off, adj = _load(nU, nV, [e[0] for e in edges], [e[1] for e in edges])
    _check_core_numbers(core, nU, nV, off, adj)
    # Lemma 1 on the example: (2,3) prunes core < 2 and keeps core >= 3
    _check_pairs(core, nU, nV, off, adj, [(2, 3), (3, 2), (1, 3), (2, 1), (3, 3)])
    core.close()


def test_random_graphs_with_isolated_vertices_and_algo_param():
    rng = np.random.default_rng(17)
    for trial in range(6):
        nU, nV = int(rng.integers(1, 400)), int(rng.integers(1, 400))
        p = float(rng.uniform(0.001, 0.05))
        mask = rng.random((nU, nV)) < p
        eu, ev = np.nonzero(mask)
        core = ABCore(0)
        core.set_param("algo", 2)  # compute prepares the core numbers itself
        core.load_edges(nU, nV, eu.astype(np.int32), ev.astype(np.int32))
        off, adj = oracle.build_csr(nU, nV, eu.astype(np.int32), ev.astype(np.int32))
        _check_pairs(core, nU, nV, off, adj, [(1, 2), (2, 2), (3, 1), (4, 4), (2, 6)])
        _check_core_numbers(core, nU, nV, off, adj)
        core.close()


def test_core_numbers_follow_a_served_update():
    (nU, nV), edges, _ = load_paper_examples()
    core, off, adj = _load(nU, nV, [e[0] for e in edges], [e[1] for e in edges])
    _check_core_numbers(core, nU, nV, off, adj)
    assert core.query_edge(4, 2, abi.ABCORE_INSERT, 1, 5) == 1
    eu = np.array([e[0] for e in edges] + [4], np.int32)
    ev = np.array([e[1] for e in edges] + [2], np.int32)
    off2, adj2 = oracle.build_csr(nU, nV, eu, ev)
    _check_core_numbers(core, nU, nV, off2, adj2)
    _check_pairs(core, nU, nV, off2, adj2, [(2, 3), (1, 5), (3, 3)])
    core.close()
