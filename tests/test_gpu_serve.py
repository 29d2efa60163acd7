"""GPU parity of on-the-fly edge queries and the serving loop against the oracle's replay.

The oracle applies the updates in order and peels the whole updated graph from scratch at every
checked step; the library answers from its scoped re-peels. Answers must match exactly, and must
not depend on how requests are batched or timed."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2606_07148_gb300 import ABCore, ABCoreError, abi
from tests.bruteforce import load_paper_examples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_07148_gb300.buildlib import build
    build()


def _reqs(stream, lo, hi):
    arr = (abi.abcore_req * (hi - lo))()
    for i, k in enumerate(range(lo, hi)):
        arr[i].op = int(stream.op[k])
        arr[i].u = int(stream.u[k])
        arr[i].v = int(stream.v[k])
        arr[i].target = int(stream.target[k])
        arr[i].tag = k
    return arr


def _serve(core, stream, targets, batch, ring=4096):
    """Submit the stream in chunks of `batch`, polling as we go; responses in sequence order."""
    import time
    core.serve_start(targets, ring_slots=ring)
    out = []
    k = 0
    n = len(stream)
    t0 = time.time()
    while k < n or len(out) < n:
        assert time.time() - t0 < 120, "serving stalled: %d submitted, %d answered" % (k, len(out))
        if k < n:
            hi = min(n, k + batch)
            seq = core.serve_submit(_reqs(stream, k, hi))
            if seq is not None:
                assert seq == list(range(k, hi))
                k = hi
        out.extend(core.serve_poll(4096))
    core.serve_stop()
    assert [r.seq for r in out] == list(range(n))
    return out


def _oracle(nU, nV, eu, ev, stream, targets, check=None):
    al = np.array([targets[t][0] for t in stream.target], dtype=np.int32)
    be = np.array([targets[t][1] for t in stream.target], dtype=np.int32)
    return oracle.replay(nU, nV, eu, ev, stream.op, stream.u, stream.v, al, be, check)


def test_paper_example1_insert_query():
    (nU, nV), edges, _ = load_paper_examples()
    eu = np.array([e[0] for e in edges], dtype=np.int32)
    ev = np.array([e[1] for e in edges], dtype=np.int32)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    assert core.query_edge(4, 2, abi.ABCORE_INSERT, 1, 5) == 1
    with pytest.raises(ABCoreError) as e:
        core.query_edge(4, 2, abi.ABCORE_INSERT, 1, 5)
    assert e.value.code == abi.ABCORE_EEXIST
    # the (2,3)-core after the insert, by the static peel on the updated graph
    mu, mv = core.compute(2, 3)
    off, adj = oracle.build_csr(nU, nV, np.append(eu, 4), np.append(ev, 2))
    wu, wv = oracle.peel(nU, nV, off, adj, 2, 3)
    assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv)
    assert core.query_edge(4, 2, abi.ABCORE_DELETE, 1, 5) == 0
    with pytest.raises(ABCoreError) as e:
        core.query_edge(4, 2, abi.ABCORE_DELETE, 1, 5)
    assert e.value.code == abi.ABCORE_ENOENT
    core.close()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_stream_small_graph_all_steps_vs_oracle(seed):
    nU, nV, m = 300, 200, 3000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.2, seed)
    eu, ev = eu.numpy(), ev.numpy()
    stream = synth.edge_update_stream(eu, ev, nU, nV, 3000, seed)
    targets = [(2, 2), (3, 3), (2, 5), (6, 6)]
    ans, bits, status = _oracle(nU, nV, eu, ev, stream, targets)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    out = _serve(core, stream, targets, batch=97)
    got = np.array([r.in_core for r in out])
    gst = np.array([r.status for r in out])
    gbits = np.array([r.u_in | (r.v_in << 1) for r in out])
    assert np.array_equal(gst, status)
    assert np.array_equal(got, ans), "first mismatch at op %d" % int(np.argmax(got != ans))
    assert np.array_equal(gbits, bits)
    # the graph left by the stream: the static peel agrees with the oracle
    al, be = 3, 2
    mu, mv = core.compute(al, be)
    cur = set(zip(eu.tolist(), ev.tolist()))
    for k in range(len(stream)):
        e = (int(stream.u[k]), int(stream.v[k]))
        if stream.op[k] == 0:
            cur.add(e)
        else:
            cur.discard(e)
    cu = np.array([e[0] for e in cur], dtype=np.int32)
    cv = np.array([e[1] for e in cur], dtype=np.int32)
    off, adj = oracle.build_csr(nU, nV, cu, cv)
    wu, wv = oracle.peel(nU, nV, off, adj, al, be)
    assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv)
    core.close()


def test_stream_answers_do_not_depend_on_batching():
    """Each result is the same alone (one request at a time, synchronous) and in the mix
    (large submissions overlapping on the device)."""
    nU, nV, m = 2000, 1000, 30000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.2, 7)
    eu, ev = eu.numpy(), ev.numpy()
    stream = synth.edge_update_stream(eu, ev, nU, nV, 1500, 7)
    targets = [(2, 2), (5, 5), (10, 20), (32, 32)]
    runs = []
    for batch in (1, 13, 1500):
        core = ABCore(0)
        core.load_edges(nU, nV, eu, ev)
        out = _serve(core, stream, targets, batch=batch, ring=2048)
        runs.append(([r.in_core for r in out], [r.status for r in out]))
        core.close()
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    alone = []
    for k in range(len(stream)):
        a, b = targets[stream.target[k]]
        try:
            alone.append((core.query_edge(int(stream.u[k]), int(stream.v[k]), int(stream.op[k]), a, b), 0))
        except ABCoreError as e:
            alone.append((None, e.code))
    core.close()
    for r in runs[1:]:
        assert r == runs[0]
    assert [s for _, s in alone] == runs[0][1]
    assert [a for a, s in alone if s == 0] == [a for a, s in zip(*runs[0]) if s == 0]
    ans, _, status = _oracle(nU, nV, eu, ev, stream, targets)
    assert runs[0][0] == ans.tolist() and runs[0][1] == status.tolist()


def test_serve_scaled_workload_vs_oracle():
    """The serving recipe scaled to 10k x 5k vertices and 200k edges; the oracle checks every
    one of the first 3000 updates and every 40th after that, over 20k updates."""
    spec = synth.WORKLOADS["serve-10kx5k-200k"]
    nU, nV, eu, ev = synth.make_graph(spec)
    eu, ev = eu.numpy(), ev.numpy()
    stream = synth.edge_update_stream(eu, ev, nU, nV, 20000, spec["seed"])
    targets = spec["targets"]
    check = np.zeros(len(stream), dtype=np.uint8)
    check[:3000] = 1
    check[3000::40] = 1
    ans, bits, status = _oracle(nU, nV, eu, ev, stream, targets, check)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    out = _serve(core, stream, targets, batch=256)
    got = np.array([r.in_core for r in out])
    gst = np.array([r.status for r in out])
    sel = check.astype(bool)
    assert np.array_equal(gst, status)
    assert np.array_equal(got[sel], ans[sel])
    core.close()


def test_serve_rejects_bad_requests():
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    core.serve_start([(2, 2)], ring_slots=8)
    bad = (abi.abcore_req * 1)()
    bad[0].op, bad[0].u, bad[0].v, bad[0].target = 0, nU, 0, 0
    with pytest.raises(ABCoreError) as e:
        core.serve_submit(bad)
    assert e.value.code == abi.ABCORE_EINVAL
    bad[0].u, bad[0].target = 0, 3
    with pytest.raises(ABCoreError) as e:
        core.serve_submit(bad)
    assert e.value.code == abi.ABCORE_EINVAL
    # ring of 8 slots: a ninth outstanding request is refused with EBUSY until responses are polled
    ok = (abi.abcore_req * 8)()
    for i in range(8):
        ok[i].op, ok[i].u, ok[i].v, ok[i].target = 1, 0, 0, 0  # deletes of (0,0): absent -> ENOENT
    eu_np, ev_np = eu.numpy(), ev.numpy()
    assert not np.any((eu_np == 0) & (ev_np == 0))
    assert core.serve_submit(ok) == list(range(8))
    assert core.serve_submit(ok) is None
    got = []
    while len(got) < 8:
        got.extend(core.serve_poll(64))
    assert all(r.status == abi.ABCORE_ENOENT for r in got)
    core.serve_stop()
    core.close()


def test_small_inserted_edge_pool_grows_and_answers_stay_exact():
    # a tiny inserted-edge pool (16 inserts' worth per target): inserts that do not fit are held
    # back until the library has grown the pool, so the whole stream -- thousands of inserts,
    # deletes of inserted edges among them -- finishes with every answer equal to the oracle's
    spec = synth.WORKLOADS["serve-10kx5k-200k"]
    nU, nV, eu, ev = synth.make_graph(spec)
    eu, ev = eu.numpy(), ev.numpy()
    stream = synth.edge_update_stream(eu, ev, nU, nV, 6000, 11)
    targets = spec["targets"]
    ans, bits, status = _oracle(nU, nV, eu, ev, stream, targets)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    core.set_param("serve_inserts", 16)
    out = _serve(core, stream, targets, batch=64, ring=128)
    assert np.array_equal(np.array([r.status for r in out]), status)
    assert np.array_equal(np.array([r.in_core for r in out]), ans)
    assert np.array_equal(np.array([r.u_in | (r.v_in << 1) for r in out]), bits)
    assert int((stream.op == 0).sum()) > 16 * 4 * 8  # far more inserts than the first pools held
    # the served graph is the oracle's final graph
    mu, mv = core.compute(5, 5)
    fin = {}
    for k in range(len(stream)):
        key = (int(stream.u[k]), int(stream.v[k]))
        fin[key] = stream.op[k] == 0
    cur = set(zip(eu.tolist(), ev.tolist()))
    for key, present in fin.items():
        (cur.add if present else cur.discard)(key)
    fu = np.array([e[0] for e in cur], dtype=np.int32)
    fv = np.array([e[1] for e in cur], dtype=np.int32)
    off, adj = oracle.build_csr(nU, nV, fu, fv)
    wu, wv = oracle.peel(nU, nV, off, adj, 5, 5)
    assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv)
    core.close()


def _query_all(core, stream, targets):
    return np.array([core.query_edge(int(stream.u[k]), int(stream.v[k]), int(stream.op[k]),
                                     targets[int(stream.target[k])][0], targets[int(stream.target[k])][1])
                     for k in range(len(stream))], dtype=np.int8)


def test_component_scope_matches_oracle_and_certificate_scope():
    # the paper's GFQ scope (the endpoints' components re-peeled from scratch) against the oracle
    # at every step and against the certificate scope of the serving loop
    spec = synth.WORKLOADS["serve-10kx5k-200k"]
    nU, nV, eu, ev = synth.make_graph(spec)
    eu, ev = eu.numpy(), ev.numpy()
    stream = synth.edge_update_stream(eu, ev, nU, nV, 1500, 5)
    targets = spec["targets"]
    ans, _, _ = _oracle(nU, nV, eu, ev, stream, targets)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    core.set_param("query_scope", 1)
    got = _query_all(core, stream, targets)
    st = core.stats()
    assert np.array_equal(got, ans)
    assert st["scope_queries"] == len(stream) and st["scope_vertices"] > 0
    core.close()
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    out = _serve(core, stream, targets, batch=128)
    assert np.array_equal(np.array([r.in_core for r in out], dtype=np.int8), got)
    core.close()


def test_component_scope_on_many_components_merging_and_splitting():
    # four disjoint random blocks: inserts bridge blocks (components merge), deletes cut bridges
    # and block edges (components split); the forest and the scoped re-peel must follow
    rng = np.random.default_rng(9)
    nb, bu, bv = 4, 30, 20
    nU, nV = nb * bu, nb * bv
    edges = set()
    for b in range(nb):
        while len(edges) < (b + 1) * 180:
            edges.add((b * bu + int(rng.integers(bu)), b * bv + int(rng.integers(bv))))
    base = sorted(edges)
    eu = np.array([e[0] for e in base], dtype=np.int32)
    ev = np.array([e[1] for e in base], dtype=np.int32)
    cur = list(base)
    ops, us, vs, tg = [], [], [], []
    present = set(base)
    for k in range(700):
        if rng.random() < 0.55:
            while True:
                u, v = int(rng.integers(nU)), int(rng.integers(nV))
                if (u, v) not in present:
                    break
            present.add((u, v)); cur.append((u, v)); ops.append(0)
        else:
            i = int(rng.integers(len(cur)))
            u, v = cur[i]
            cur[i] = cur[-1]; cur.pop(); present.discard((u, v)); ops.append(1)
        us.append(u); vs.append(v); tg.append(int(rng.integers(3)))
    stream = synth.StreamOp(op=np.array(ops, np.int8), u=np.array(us, np.int32), v=np.array(vs, np.int32),
                            target=np.array(tg, np.int8), t_unit=np.arange(len(ops), dtype=np.float64))
    targets = [(2, 2), (3, 4), (5, 3)]
    ans, _, _ = _oracle(nU, nV, eu, ev, stream, targets)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    core.set_param("query_scope", 1)
    got = _query_all(core, stream, targets)
    assert np.array_equal(got, ans)
    # the forest after all updates names the oracle's components of the final graph
    lu, lv, ncomp = core.components()
    fu = np.array([e[0] for e in cur], dtype=np.int32)
    fv = np.array([e[1] for e in cur], dtype=np.int32)
    off, adj = oracle.build_csr(nU, nV, fu, fv)
    lab, nc = oracle.components(nU, nV, off, adj)
    assert ncomp == nc and np.array_equal(np.concatenate([lu.cpu().numpy(), lv.cpu().numpy()]), lab)
    core.close()
