"""GPU parity of the query helpers against the oracle: alpha_offset and the paper's default
query (Section 6), and community search (the Remark after GFQ, Section 5)."""

import numpy as np
import pytest

import oracle
import synth
from paper_2606_07148_gb300 import ABCore, ABCoreError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_07148_gb300.buildlib import build
    build()


@pytest.fixture(scope="module")
def small():
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    eu, ev = eu.numpy(), ev.numpy()
    off, adj = oracle.build_csr(nU, nV, eu, ev)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    yield nU, nV, eu, ev, off, adj, core
    core.close()


def _oracle_offset(nU, nV, off, adj, alpha):
    # alpha >= 1: once no lower vertex is left no upper one is, so the scan ends by the largest
    # lower degree
    assert alpha >= 1
    best = 0
    for b in range(1, int(np.diff(off[nU:]).max()) + 2):
        wu, wv = oracle.peel(nU, nV, off, adj, alpha, b)
        if wu.sum() + wv.sum() == 0:
            break
        best = b
    return best


def test_alpha_offset_and_default_query(small):
    nU, nV, eu, ev, off, adj, core = small
    for alpha in (1, 2, 3, 5, 8):
        assert core.alpha_offset(alpha) == _oracle_offset(nU, nV, off, adj, alpha), alpha
    with pytest.raises(ABCoreError):
        core.alpha_offset(0)
    # the library computes the whole default query; the oracle restates it from the paper
    assert core.default_query() == oracle.default_query(nU, nV, off, adj)


@pytest.mark.parametrize("a,b", [(5, 7), (7, 5), (3, 3), (12, 2), (1, 9)])
def test_default_query_complete_bipartite_matches_oracle(a, b):
    # K_{a,b}: every (alpha, beta)-core with alpha <= b and beta <= a is the whole graph
    uu, vv = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
    eu, ev = uu.ravel().astype(np.int32), vv.ravel().astype(np.int32)
    off, adj = oracle.build_csr(a, b, eu, ev)
    core = ABCore(0)
    core.load_edges(a, b, eu, ev)
    got = core.default_query()
    core.close()
    assert got == oracle.default_query(a, b, off, adj)


def _oracle_community(nU, nV, off, adj, eu, ev, q, alpha, beta):
    wu, wv = oracle.peel(nU, nV, off, adj, alpha, beta)
    inside = np.concatenate([wu, wv]).astype(bool)
    if not inside[q]:
        return np.zeros(nU + nV, np.uint8)
    keep = inside[eu] & inside[nU + ev]
    o2, a2 = oracle.build_csr(nU, nV, eu[keep], ev[keep])
    lab, _ = oracle.components(nU, nV, o2, a2)
    return ((lab == lab[q]) & inside).astype(np.uint8)


def test_community_search(small):
    nU, nV, eu, ev, off, adj, core = small
    rng = np.random.default_rng(3)
    for alpha, beta in [(1, 1), (2, 2), (2, 3), (3, 5), (1, 4)]:
        for _ in range(4):
            layer = int(rng.integers(2))
            vid = int(rng.integers(nU if layer == 0 else nV))
            q = vid if layer == 0 else nU + vid
            want = _oracle_community(nU, nV, off, adj, eu, ev, q, alpha, beta)
            mu, mv, size = core.community(layer, vid, alpha, beta)
            got = np.concatenate([mu.cpu().numpy(), mv.cpu().numpy()])
            assert np.array_equal(got, want), (alpha, beta, layer, vid)
            assert size == int(want.sum())
    # a host-buffer call, and a bad layer
    hu, hv = np.zeros(nU, np.uint8), np.zeros(nV, np.uint8)
    _, _, size = core.community(0, 0, 1, 1, hu, hv)
    want = _oracle_community(nU, nV, off, adj, eu, ev, 0, 1, 1)
    assert np.array_equal(np.concatenate([hu, hv]), want) and size == int(want.sum())
    with pytest.raises(ABCoreError):
        core.community(2, 0, 1, 1)
