"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test ties the oracle to the paper's definitions through an independent route: brute-force
subset enumeration (Definition 1 read literally), closed forms, networkx's k-core code
(Definition 2 and the (k,k) special case), Lemma 1, the nested property, the fixpoint invariant
and the worked examples printed in the paper.
"""

import itertools
import random

import networkx as nx
import numpy as np
import pytest

import oracle
from tests.bruteforce import load_paper_examples, mask_from_bits, max_feasible


def _peel_edges(nU, nV, edges, a, b):
    eu = np.array([e[0] for e in edges], dtype=np.int32)
    ev = np.array([e[1] for e in edges], dtype=np.int32)
    off, adj = oracle.build_csr(nU, nV, eu, ev)
    return oracle.peel(nU, nV, off, adj, a, b)


def _random_graph(rng, nU, nV, p):
    return [(u, v) for u in range(nU) for v in range(nV) if rng.random() < p]


# ------------------------------------------------------------------------------------------
# CSR storage
# ------------------------------------------------------------------------------------------
def test_csr_rows_match_direct_construction():
    rng = random.Random(11)
    for _ in range(20):
        nU, nV = rng.randint(0, 30), rng.randint(0, 30)
        edges = _random_graph(rng, nU, nV, rng.random() * 0.5)
        rng.shuffle(edges)
        eu = np.array([e[0] for e in edges], dtype=np.int32)
        ev = np.array([e[1] for e in edges], dtype=np.int32)
        off, adj = oracle.build_csr(nU, nV, eu, ev)
        assert off[0] == 0 and off[-1] == 2 * len(edges)
        for u in range(nU):
            want = sorted(nU + v for (x, v) in edges if x == u)
            assert list(adj[off[u]:off[u + 1]]) == want
        for v in range(nV):
            want = sorted(u for (u, y) in edges if y == v)
            assert list(adj[off[nU + v]:off[nU + v + 1]]) == want


def test_csr_rejects_duplicates_and_out_of_range():
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_csr(2, 2, np.array([0, 0]), np.array([1, 1]))
    assert e.value.code == -4
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_csr(2, 2, np.array([0, 2]), np.array([1, 1]))
    assert e.value.code == -1
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_csr(2, 2, np.array([0]), np.array([-1]))
    assert e.value.code == -1


# ------------------------------------------------------------------------------------------
# Definition 1 by brute force
# ------------------------------------------------------------------------------------------
def test_bruteforce_every_graph_up_to_3x3():
    """Every bipartite graph with |U|, |V| <= 3 and every (alpha, beta) in [0, 4]^2."""
    count = 0
    for nU in range(0, 4):
        for nV in range(0, 4):
            pairs = [(u, v) for u in range(nU) for v in range(nV)]
            for sel in range(1 << len(pairs)):
                edges = [p for i, p in enumerate(pairs) if sel >> i & 1]
                for a in range(5):
                    for b in range(5):
                        want = mask_from_bits(max_feasible(nU, nV, edges, a, b), nU, nV)
                        got = _peel_edges(nU, nV, edges, a, b)
                        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), \
                            (nU, nV, edges, a, b)
                        count += 1
    assert count == sum(25 * (1 << (u * v)) for u in range(4) for v in range(4))


def test_bruteforce_random_graphs_up_to_14_vertices():
    rng = random.Random(7)
    for _ in range(60):
        nU = rng.randint(1, 8)
        nV = rng.randint(1, 14 - nU)
        edges = _random_graph(rng, nU, nV, rng.uniform(0.2, 0.8))
        a, b = rng.randint(0, 5), rng.randint(0, 5)
        want = mask_from_bits(max_feasible(nU, nV, edges, a, b), nU, nV)
        got = _peel_edges(nU, nV, edges, a, b)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (nU, nV, edges, a, b)


# ------------------------------------------------------------------------------------------
# Closed forms
# ------------------------------------------------------------------------------------------
def test_zero_thresholds_keep_every_vertex_including_isolated():
    edges = [(0, 0), (1, 0)]
    mu, mv = _peel_edges(4, 3, edges, 0, 0)
    assert mu.tolist() == [1, 1, 1, 1] and mv.tolist() == [1, 1, 1]


def test_alpha_one_closed_form():
    """(1, beta): V part = {v : deg(v) >= beta}; U part = {u : some neighbour has deg >= beta}."""
    rng = random.Random(3)
    for _ in range(30):
        nU, nV = rng.randint(1, 40), rng.randint(1, 40)
        edges = _random_graph(rng, nU, nV, rng.uniform(0.02, 0.3))
        degv = np.zeros(nV, dtype=int)
        for _, v in edges:
            degv[v] += 1
        for b in range(1, 8):
            mu, mv = _peel_edges(nU, nV, edges, 1, b)
            want_v = (degv >= b).astype(np.uint8)
            want_u = np.zeros(nU, dtype=np.uint8)
            for u, v in edges:
                if degv[v] >= b:
                    want_u[u] = 1
            assert np.array_equal(mv, want_v) and np.array_equal(mu, want_u)


def test_beta_one_closed_form():
    rng = random.Random(4)
    for _ in range(30):
        nU, nV = rng.randint(1, 40), rng.randint(1, 40)
        edges = _random_graph(rng, nU, nV, rng.uniform(0.02, 0.3))
        degu = np.zeros(nU, dtype=int)
        for u, _ in edges:
            degu[u] += 1
        for a in range(1, 8):
            mu, mv = _peel_edges(nU, nV, edges, a, 1)
            want_u = (degu >= a).astype(np.uint8)
            want_v = np.zeros(nV, dtype=np.uint8)
            for u, v in edges:
                if degu[u] >= a:
                    want_v[v] = 1
            assert np.array_equal(mu, want_u) and np.array_equal(mv, want_v)


def test_complete_bipartite():
    for a_n in range(1, 6):
        for b_n in range(1, 6):
            edges = [(u, v) for u in range(a_n) for v in range(b_n)]
            for a in range(1, 7):
                for b in range(1, 7):
                    mu, mv = _peel_edges(a_n, b_n, edges, a, b)
                    full = a <= b_n and b <= a_n
                    assert mu.all() == full and mv.all() == full
                    assert (mu.any() or mv.any()) == full
            # a zero threshold keeps its whole layer; the other layer then sees every vertex
            for b in range(0, 7):
                mu, mv = _peel_edges(a_n, b_n, edges, 0, b)
                assert mu.all() and mv.all() == (b <= a_n) and mv.any() == (b <= a_n)
            for a in range(0, 7):
                mu, mv = _peel_edges(a_n, b_n, edges, a, 0)
                assert mv.all() and mu.all() == (a <= b_n) and mu.any() == (a <= b_n)


def test_forest_has_empty_2_2_core():
    rng = random.Random(5)
    for _ in range(20):
        g = nx.random_labeled_tree(rng.randint(2, 40), seed=rng.randint(0, 10**6))
        side = nx.bipartite.color(g)
        U = sorted(x for x in g if side[x] == 0)
        V = sorted(x for x in g if side[x] == 1)
        iu = {x: i for i, x in enumerate(U)}
        iv = {x: i for i, x in enumerate(V)}
        edges = [(iu[x], iv[y]) if side[x] == 0 else (iu[y], iv[x]) for x, y in g.edges]
        mu, mv = _peel_edges(len(U), len(V), edges, 2, 2)
        assert not mu.any() and not mv.any()


def test_even_cycle():
    for k in range(2, 12):
        edges = [(i, i) for i in range(k)] + [(i, (i + 1) % k) for i in range(k)]
        mu, mv = _peel_edges(k, k, edges, 2, 2)
        assert mu.all() and mv.all()
        mu, mv = _peel_edges(k, k, edges, 2, 3)
        assert not mu.any() and not mv.any()


# ------------------------------------------------------------------------------------------
# Definition 2 and the (k,k) special case, against networkx
# ------------------------------------------------------------------------------------------
def _nx_graph(nU, nV, eu, ev):
    g = nx.Graph()
    g.add_nodes_from(range(nU + nV))
    g.add_edges_from(zip(eu.tolist(), (ev + nU).tolist()))
    return g


def test_kk_core_and_core_numbers_match_networkx():
    import synth
    eu, ev = synth.chung_lu_edges(600, 400, 5000, 2.2, 2.4, seed=9)
    eu, ev = eu.numpy(), ev.numpy()
    off, adj = oracle.build_csr(600, 400, eu, ev)
    g = _nx_graph(600, 400, eu, ev)
    want = nx.core_number(g)
    core = oracle.core_numbers(600, 400, off, adj)
    assert all(core[x] == want[x] for x in range(1000))
    for k in range(0, max(want.values()) + 2):
        mu, mv = oracle.peel(600, 400, off, adj, k, k)
        got = set(np.nonzero(np.concatenate([mu, mv]))[0].tolist())
        kc = set(nx.k_core(g, k).nodes) if k > 0 else set(range(1000))
        assert got == kc, k


# ------------------------------------------------------------------------------------------
# Invariants on Chung-Lu graphs: fixpoint, maximality by re-peel, nested property, Lemma 1
# ------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cl_graph():
    import synth
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    eu, ev = eu.numpy(), ev.numpy()
    off, adj = oracle.build_csr(nU, nV, eu, ev)
    return nU, nV, eu, ev, off, adj


def test_fixpoint_and_repeel_identity(cl_graph):
    nU, nV, eu, ev, off, adj = cl_graph
    for a, b in [(2, 3), (1, 1), (3, 2), (5, 5), (2, 10), (10, 2), (7, 4)]:
        mu, mv = oracle.peel(nU, nV, off, adj, a, b)
        alive = np.concatenate([mu, mv]).astype(bool)
        for x in np.nonzero(alive)[0]:
            nb = adj[off[x]:off[x + 1]]
            thr = a if x < nU else b
            assert alive[nb].sum() >= thr
        keep = alive[eu] & alive[nU + ev]
        off2, adj2 = oracle.build_csr(nU, nV, eu[keep], ev[keep])
        mu2, mv2 = oracle.peel(nU, nV, off2, adj2, a, b)
        assert np.array_equal(np.concatenate([mu2, mv2]).astype(bool), alive)


def test_nested_property(cl_graph):
    nU, nV, eu, ev, off, adj = cl_graph
    vals = [0, 1, 2, 3, 5, 8]
    masks = {(a, b): np.concatenate(oracle.peel(nU, nV, off, adj, a, b)) for a in vals for b in vals}
    for (a, b), (a2, b2) in itertools.product(masks, masks):
        if a2 >= a and b2 >= b:
            assert np.all(masks[(a2, b2)] <= masks[(a, b)])


def test_lemma1_pruning_bounds(cl_graph):
    nU, nV, eu, ev, off, adj = cl_graph
    g = _nx_graph(nU, nV, eu, ev)
    core = nx.core_number(g)
    c = np.array([core[x] for x in range(nU + nV)])
    for a, b in [(2, 3), (3, 2), (2, 6), (6, 2), (4, 4), (1, 5)]:
        alive = np.concatenate(oracle.peel(nU, nV, off, adj, a, b)).astype(bool)
        assert not alive[c < min(a, b)].any()
        assert alive[c >= max(a, b)].all()


# ------------------------------------------------------------------------------------------
# The paper's worked examples
# ------------------------------------------------------------------------------------------
def test_paper_worked_examples():
    (nU, nV), edges, steps = load_paper_examples()
    assert nU + nV == 15 and len(edges) == 20
    edges = list(edges)
    for step in steps:
        eu = np.array([e[0] for e in edges], dtype=np.int32)
        ev = np.array([e[1] for e in edges], dtype=np.int32)
        off, adj = oracle.build_csr(nU, nV, eu, ev)
        if step[0] == "core":
            _, a, b, us, vs = step
            mu, mv = oracle.peel(nU, nV, off, adj, a, b)
            assert np.nonzero(mu)[0].tolist() == us and np.nonzero(mv)[0].tolist() == vs, (a, b)
            bf = mask_from_bits(max_feasible(nU, nV, edges, a, b), nU, nV)
            assert np.array_equal(bf[0], mu) and np.array_equal(bf[1], mv)
        elif step[0] == "corenum":
            assert oracle.core_numbers(nU, nV, off, adj).tolist() == step[1]
        elif step[0] == "insert":
            u, v = step[1], step[2]
            assert sum(1 for e in edges if e[1] == v) == 4  # deg(v2) = 4 before the insert
            edges.append((u, v))


def test_paper_example2_first_round():
    """(1,3): exactly v3, v5, v6 violate at the start, and they are the only vertices removed."""
    (nU, nV), edges, _ = load_paper_examples()
    degv = [sum(1 for e in edges if e[1] == v) for v in range(nV)]
    assert [v for v in range(nV) if degv[v] < 3] == [3, 5, 6]
    eu = np.array([e[0] for e in edges], dtype=np.int32)
    ev = np.array([e[1] for e in edges], dtype=np.int32)
    off, adj = oracle.build_csr(nU, nV, eu, ev)
    mu, mv = oracle.peel(nU, nV, off, adj, 1, 3)
    assert mu.all() and np.nonzero(1 - mv)[0].tolist() == [3, 5, 6]


# ------------------------------------------------------------------------------------------
# On-the-fly queries: the replay against brute force on tiny streams
# ------------------------------------------------------------------------------------------
def test_replay_matches_bruteforce():
    rng = random.Random(21)
    for _ in range(25):
        nU, nV = rng.randint(1, 6), rng.randint(1, 6)
        edges = _random_graph(rng, nU, nV, 0.4)
        cur = set(edges)
        ops, qu, qv, al, be, want, wstat = [], [], [], [], [], [], []
        for _ in range(12):
            u, v = rng.randrange(nU), rng.randrange(nV)
            op = rng.randrange(2)
            a, b = rng.randint(1, 4), rng.randint(1, 4)
            status = 0
            if op == 0:
                if (u, v) in cur:
                    status = -4
                else:
                    cur.add((u, v))
            else:
                if (u, v) not in cur:
                    status = -5
                else:
                    cur.discard((u, v))
            bits = max_feasible(nU, nV, sorted(cur), a, b)
            ans = int((bits >> u) & 1 and (bits >> (nU + v)) & 1)
            ops.append(op); qu.append(u); qv.append(v); al.append(a); be.append(b)
            want.append(ans); wstat.append(status)
        eu = np.array([e[0] for e in edges], dtype=np.int32)
        ev = np.array([e[1] for e in edges], dtype=np.int32)
        ans, bits, status = oracle.replay(nU, nV, eu, ev, ops, qu, qv, al, be)
        assert ans.tolist() == want
        assert status.tolist() == wstat


def test_replay_paper_example1_insert():
    """Example 1: after inserting (u4, v2), the edge lies in the (1,5)-core."""
    (nU, nV), edges, _ = load_paper_examples()
    eu = np.array([e[0] for e in edges], dtype=np.int32)
    ev = np.array([e[1] for e in edges], dtype=np.int32)
    ans, bits, status = oracle.replay(nU, nV, eu, ev, [0], [4], [2], [1], [5])
    assert ans.tolist() == [1] and bits.tolist() == [3] and status.tolist() == [0]


# ------------------------------------------------------------------------------------------
# Connected components (the labels GFQ keeps, Section 5)
# ------------------------------------------------------------------------------------------
def _components_edges(nU, nV, edges):
    eu = np.array([e[0] for e in edges], dtype=np.int32)
    ev = np.array([e[1] for e in edges], dtype=np.int32)
    off, adj = oracle.build_csr(nU, nV, eu, ev)
    return oracle.components(nU, nV, off, adj)


def test_components_match_scipy():
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    rng = random.Random(23)
    for _ in range(40):
        nU, nV = rng.randint(0, 40), rng.randint(0, 40)
        edges = _random_graph(rng, nU, nV, rng.random() * 0.08)
        lab, nc = _components_edges(nU, nV, edges)
        n = nU + nV
        rows = [u for u, v in edges] + [nU + v for u, v in edges]
        cols = [nU + v for u, v in edges] + [u for u, v in edges]
        A = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
        k, sl = connected_components(A, directed=False)
        assert nc == k
        # same partition, and each label is the smallest id of its component
        for c in range(k):
            members = np.nonzero(sl == c)[0]
            assert set(lab[members].tolist()) == {int(members.min())}


def test_components_closed_forms():
    lab, nc = _components_edges(3, 4, [])                        # no edges: every vertex alone
    assert nc == 7 and list(lab) == list(range(7))
    lab, nc = _components_edges(3, 4, [(u, v) for u in range(3) for v in range(4)])
    assert nc == 1 and set(lab.tolist()) == {0}                  # complete bipartite
    lab, nc = _components_edges(5, 5, [(i, i) for i in range(5)])
    assert nc == 5 and list(lab) == [0, 1, 2, 3, 4, 0, 1, 2, 3, 4]   # perfect matching
    # path u0 - v0 - u1 - v1 - u2 plus an isolated v2
    lab, nc = _components_edges(3, 3, [(0, 0), (1, 0), (1, 1), (2, 1)])
    assert nc == 2 and list(lab) == [0, 0, 0, 0, 0, 5]


# ------------------------------------------------------------------------------------------
# The paper's default query (Section 6)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("a,b", [(5, 7), (7, 5), (3, 3), (12, 2), (1, 9), (10, 10)])
def test_default_query_complete_bipartite_closed_form(a, b):
    # K_{a,b} (|U| = a, |L| = b): the k-core numbers are all min(a, b), and an (alpha, beta)-core
    # with alpha <= b is the whole graph for beta <= a and empty beyond, so alpha_offset = a
    edges = [(u, v) for u in range(a) for v in range(b)]
    eu = np.array([e[0] for e in edges], dtype=np.int32)
    ev = np.array([e[1] for e in edges], dtype=np.int32)
    off, adj = oracle.build_csr(a, b, eu, ev)
    delta, alpha, offset, beta = oracle.default_query(a, b, off, adj)
    assert delta == min(a, b)
    assert alpha == max(1, (2 * min(a, b)) // 5)
    assert offset == a
    assert beta == (3 * a) // 5


def test_default_query_offset_by_brute_force():
    # alpha_offset checked against subset enumeration (Definition 1 read literally) for every
    # beta, and delta against networkx's core numbers
    rng = random.Random(17)
    for trial in range(12):
        nU, nV = rng.randint(2, 6), rng.randint(2, 6)
        edges = _random_graph(rng, nU, nV, 0.6)
        eu = np.array([e[0] for e in edges], dtype=np.int32)
        ev = np.array([e[1] for e in edges], dtype=np.int32)
        off, adj = oracle.build_csr(nU, nV, eu, ev)
        delta, alpha, offset, beta = oracle.default_query(nU, nV, off, adj)
        G = nx.Graph()
        G.add_nodes_from(range(nU + nV))
        G.add_edges_from((u, nU + v) for u, v in edges)
        assert delta == max(nx.core_number(G).values())
        want = 0
        for bb in range(1, nU + 2):
            if max_feasible(nU, nV, edges, alpha, bb):
                want = bb
        assert offset == want, (trial, edges)
        assert beta == (3 * want) // 5
