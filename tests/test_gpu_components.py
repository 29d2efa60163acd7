"""GPU parity of the connected-components labels (the labels GFQ keeps, Section 5) against the
oracle's breadth-first search, on static graphs and on graphs changed by served updates."""

import time

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2606_07148_gb300 import ABCore, abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_07148_gb300.buildlib import build
    build()


def _oracle_labels(nU, nV, eu, ev):
    off, adj = oracle.build_csr(nU, nV, np.asarray(eu, np.int32), np.asarray(ev, np.int32))
    return oracle.components(nU, nV, off, adj)


def _check(core, nU, nV, eu, ev, host=False):
    want, wn = _oracle_labels(nU, nV, eu, ev)
    if host:
        lu = np.zeros(nU, np.int32)
        lv = np.zeros(nV, np.int32)
        _, _, nc = core.components(lu, lv)
    else:
        tu, tv, nc = core.components()
        lu, lv = tu.cpu().numpy(), tv.cpu().numpy()
    assert nc == wn
    assert np.array_equal(lu, want[:nU]) and np.array_equal(lv, want[nU:])


def test_components_small_chung_lu():
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    _check(core, nU, nV, eu.numpy(), ev.numpy())
    _check(core, nU, nV, eu.numpy(), ev.numpy(), host=True)
    core.close()


def test_components_every_row_class_and_isolated_vertices():
    # hub rows (>= 1024 entries: a block each), medium rows (>= 32: a warp each), short rows
    # (a thread each), isolated vertices on both layers, and several components
    rng = np.random.default_rng(5)
    nU, nV = 3000, 2500
    edges = set()
    for v in range(0, 2000):                 # hub u0 joins v0..v1999
        edges.add((0, v))
    for u in range(1, 40):                   # medium rows u1..u39: 40 random v in 0..1999
        for v in rng.choice(2000, 40, replace=False):
            edges.add((u, int(v)))
    for u in range(40, 2000):                # short rows: pairs among v2000..v2399, own components
        edges.add((u, 2000 + (u % 400)))
    # u2000..2999 and v2400..2499 stay isolated
    eu = np.array([e[0] for e in edges], np.int32)
    ev = np.array([e[1] for e in edges], np.int32)
    core = ABCore(0)
    core.load_edges(nU, nV, torch.from_numpy(eu).cuda(), torch.from_numpy(ev).cuda())
    _check(core, nU, nV, eu, ev)
    core.close()


def test_components_empty_and_edgeless():
    core = ABCore(0)
    core.load_edges(4, 3, np.zeros(0, np.int32), np.zeros(0, np.int32))
    _check(core, 4, 3, [], [])
    core.close()


def _reqs(ops, us, vs):
    arr = (abi.abcore_req * len(ops))()
    for i, (o, u, v) in enumerate(zip(ops, us, vs)):
        arr[i].op, arr[i].u, arr[i].v, arr[i].target, arr[i].tag = int(o), int(u), int(v), 0, i
    return arr


def _serve_all(core, ops, us, vs):
    seq = core.serve_submit(_reqs(ops, us, vs))
    assert seq is not None
    got = []
    t0 = time.time()
    while len(got) < len(ops):
        assert time.time() - t0 < 60
        got.extend(core.serve_poll(4096))
    return got


def test_components_follow_served_inserts_and_deletes():
    spec = dict(synth.WORKLOADS["serve-10kx5k-200k"])
    nU, nV, eu, ev = synth.make_graph(spec)
    eu, ev = eu.numpy(), ev.numpy()
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    core.serve_start([(2, 2)], ring_slots=8192)
    edges = set(zip(eu.tolist(), ev.tolist()))
    rng = np.random.default_rng(9)
    ins = []
    while len(ins) < 300:
        u, v = int(rng.integers(nU)), int(rng.integers(nV))
        if (u, v) not in edges:
            edges.add((u, v))
            ins.append((u, v))
    got = _serve_all(core, [abi.ABCORE_INSERT] * len(ins), [e[0] for e in ins], [e[1] for e in ins])
    assert all(r.status == abi.ABCORE_OK for r in got)
    cur = sorted(edges)
    _check(core, nU, nV, [e[0] for e in cur], [e[1] for e in cur])
    # deletes may split components; then a few more inserts
    dels = [cur[i] for i in rng.choice(len(cur), 2000, replace=False)]
    for e in dels:
        edges.discard(e)
    got = _serve_all(core, [abi.ABCORE_DELETE] * len(dels), [e[0] for e in dels], [e[1] for e in dels])
    assert all(r.status == abi.ABCORE_OK for r in got)
    cur = sorted(edges)
    _check(core, nU, nV, [e[0] for e in cur], [e[1] for e in cur])
    more = []
    while len(more) < 100:
        u, v = int(rng.integers(nU)), int(rng.integers(nV))
        if (u, v) not in edges:
            edges.add((u, v))
            more.append((u, v))
    _serve_all(core, [abi.ABCORE_INSERT] * len(more), [e[0] for e in more], [e[1] for e in more])
    cur = sorted(edges)
    _check(core, nU, nV, [e[0] for e in cur], [e[1] for e in cur], host=True)
    core.serve_stop()
    core.close()
