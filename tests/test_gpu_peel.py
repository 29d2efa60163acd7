"""GPU parity of the device CSR builder and the single (alpha, beta)-core peel against the oracle.

Masks are integer results, so the bar is bit-exact equality with the oracle on the same seeded
input. Every call goes through the C ABI (paper_2606_07148_gb300.abi via the ABCore wrapper).
"""

import random

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2606_07148_gb300 import ABCore, ABCoreError, abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_07148_gb300.buildlib import build
    build()


def _np(t):
    return t.cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)


def _check_pairs(core, nU, nV, eu, ev, pairs, off=None, adj=None):
    if off is None:
        off, adj = oracle.build_csr(nU, nV, _np(eu), _np(ev))
    for a, b in pairs:
        mu, mv = core.compute(a, b)
        wu, wv = oracle.peel(nU, nV, off, adj, a, b)
        gu, gv = _np(mu), _np(mv)
        assert np.array_equal(gu, wu) and np.array_equal(gv, wv), \
            "(%d,%d): U diff %d, V diff %d" % (a, b, int((gu != wu).sum()), int((gv != wv).sum()))


# ------------------------------------------------------------------------------------------
# device CSR builder
# ------------------------------------------------------------------------------------------
def _check_export(core, nU, nV, eu, ev):
    off, adj, n2o = core.export_csr()
    o_off, o_adj = oracle.build_csr(nU, nV, _np(eu), _np(ev))
    n = nU + nV
    assert off[0] == 0 and off[n] == 2 * len(_np(eu))
    assert sorted(n2o[:nU].tolist()) == list(range(nU))
    assert sorted(n2o[nU:].tolist()) == list(range(nV))
    deg = np.diff(off)
    assert np.all(np.diff(deg[:nU]) <= 0) and np.all(np.diff(deg[nU:]) <= 0)
    old_unified = np.concatenate([n2o[:nU], n2o[nU:] + nU]).astype(np.int64)
    for x in range(n):
        row = adj[off[x]:off[x + 1]]
        assert np.all(np.diff(row) > 0)
        if x < nU:
            assert np.all((row >= nU) & (row < n))
        else:
            assert np.all((row >= 0) & (row < nU))
        ox = old_unified[x]
        want = o_adj[o_off[ox]:o_off[ox + 1]]
        assert np.array_equal(np.sort(old_unified[row]), want)


def test_csr_builder_matches_oracle():
    core = ABCore(0)
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    _check_export(core, nU, nV, eu, ev)
    rng = random.Random(3)
    for _ in range(6):
        nU, nV = rng.randint(1, 300), rng.randint(1, 300)
        m = rng.randint(0, min(nU * nV, 3000))
        eu, ev = synth.chung_lu_edges(nU, nV, m, 2.2, 2.2, rng.randint(0, 999)) if m else (
            torch.zeros(0, dtype=torch.int32), torch.zeros(0, dtype=torch.int32))
        core.load_edges(nU, nV, eu, ev)  # host pointers
        _check_export(core, nU, nV, eu, ev)
    core.close()


def test_csr_builder_rejects_bad_input():
    core = ABCore(0)
    with pytest.raises(ABCoreError) as e:
        core.load_edges(3, 3, np.array([0, 1, 0]), np.array([1, 2, 1]))
    assert e.value.code == abi.ABCORE_EEXIST
    with pytest.raises(ABCoreError) as e:
        core.load_edges(3, 3, np.array([0, 3]), np.array([1, 2]))
    assert e.value.code == abi.ABCORE_EINVAL
    with pytest.raises(ABCoreError) as e:
        core.load_edges(3, 3, np.array([0, 1]), np.array([-1, 2]))
    assert e.value.code == abi.ABCORE_EINVAL
    with pytest.raises(ABCoreError) as e:
        core.compute(1, 1)
    assert e.value.code == abi.ABCORE_ENOTLOADED
    core.load_edges(3, 3, np.array([0, 1]), np.array([1, 2]))
    with pytest.raises(ABCoreError) as e:
        core.compute(-1, 1)
    assert e.value.code == abi.ABCORE_EINVAL
    core.close()


def test_load_csr_and_validation():
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
    m = len(eu)
    offU, adjU = off[:nU + 1], adj[:m] - nU
    offV, adjV = off[nU:] - m, adj[m:]
    core = ABCore(0)
    core.load_csr(nU, nV, offU, adjU, offV, adjV, validate=True)
    _check_pairs(core, nU, nV, eu, ev, [(2, 3), (4, 4)], off, adj)
    bad = adjV.copy()
    bad[0], bad[-1] = bad[-1], bad[0]
    if not np.array_equal(bad, adjV):
        with pytest.raises(ABCoreError) as e:
            core.load_csr(nU, nV, offU, adjU, offV, bad, validate=True)
        assert e.value.code == abi.ABCORE_EINVAL
    bad_off = offU.copy()
    bad_off[1], bad_off[2] = bad_off[2] + 5, bad_off[1]
    with pytest.raises(ABCoreError):
        core.load_csr(nU, nV, bad_off, adjU)
    core.close()


# ------------------------------------------------------------------------------------------
# the peel
# ------------------------------------------------------------------------------------------
PAIRS_SMALL = [(a, b) for a in (0, 1, 2, 3, 5, 8, 13, 40, 250) for b in (0, 1, 2, 3, 4, 7, 21, 300)]


@pytest.mark.parametrize("mode", [-1, 0, 1, 2, 3])
@pytest.mark.parametrize("chunk", [32, 1024])
def test_peel_small_graph_all_modes(mode, chunk):
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    core = ABCore(0)
    core.set_param("mode", mode)
    core.set_param("chunk", chunk)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    _check_pairs(core, nU, nV, eu, ev, PAIRS_SMALL)
    core.close()


def test_peel_tiny_random_graphs():
    rng = random.Random(17)
    core = ABCore(0)
    for _ in range(40):
        nU, nV = rng.randint(1, 12), rng.randint(1, 12)
        edges = [(u, v) for u in range(nU) for v in range(nV) if rng.random() < rng.uniform(0.1, 0.9)]
        eu = np.array([e[0] for e in edges], dtype=np.int32)
        ev = np.array([e[1] for e in edges], dtype=np.int32)
        core.load_edges(nU, nV, eu, ev)
        core.set_param("mode", rng.randint(-1, 3))
        _check_pairs(core, nU, nV, eu, ev, [(rng.randint(0, 6), rng.randint(0, 6)) for _ in range(6)])
    core.close()


def test_peel_edge_cases():
    core = ABCore(0)
    # no edges: a vertex survives only if its layer's threshold is 0
    core.load_edges(5, 4, np.zeros(0, np.int32), np.zeros(0, np.int32))
    for a, b in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        mu, mv = core.compute(a, b)
        assert _np(mu).tolist() == [int(a == 0)] * 5 and _np(mv).tolist() == [int(b == 0)] * 4
    # empty layers
    core.load_edges(0, 3, np.zeros(0, np.int32), np.zeros(0, np.int32))
    mu, mv = core.compute(0, 0)
    assert _np(mv).tolist() == [1, 1, 1]
    # complete bipartite K_{4,6} with isolated extras
    eu = np.repeat(np.arange(4), 6).astype(np.int32)
    ev = np.tile(np.arange(6), 4).astype(np.int32)
    core.load_edges(7, 9, eu, ev)
    _check_pairs(core, 7, 9, eu, ev, [(a, b) for a in range(0, 8) for b in range(0, 6)] + [(10**6, 1), (1, 10**6)])
    core.close()


def test_host_and_device_pointers_and_async_agree():
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
    core = ABCore(0)
    core.load_edges(nU, nV, eu.numpy(), ev.numpy())
    pairs = [(2, 3), (3, 3), (1, 7), (6, 2), (9, 9)]
    outs = []
    for a, b in pairs:
        hu = np.zeros(nU, np.uint8)
        hv = np.zeros(nV, np.uint8)
        core.compute(a, b, hu, hv)
        du = torch.empty(nU, dtype=torch.uint8, device="cuda")
        dv = torch.empty(nV, dtype=torch.uint8, device="cuda")
        core.compute(a, b, du, dv, asynchronous=True)
        outs.append((du, dv, hu, hv))
    core.sync()
    for (a, b), (du, dv, hu, hv) in zip(pairs, outs):
        wu, wv = oracle.peel(nU, nV, off, adj, a, b)
        assert np.array_equal(hu, wu) and np.array_equal(hv, wv)
        assert np.array_equal(_np(du), wu) and np.array_equal(_np(dv), wv)
    core.close()


def test_bounded_wait_reports_timeout_and_context_recovers():
    """A queue slot that nothing fills makes the cascade's bounded wait expire: the call returns
    ABCORE_ETIMEDOUT, and the next call on the same context is correct."""
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    core.set_param("timeout_ms", 50)
    core.set_param("debug_stall_slots", 1)
    with pytest.raises(ABCoreError) as e:
        core.compute(2, 3)
    assert e.value.code == abi.ABCORE_ETIMEDOUT
    core.set_param("debug_stall_slots", 0)
    core.set_param("timeout_ms", 4000)
    _check_pairs(core, nU, nV, eu, ev, [(2, 3), (5, 5)])
    core.close()


def test_peel_mid_size_power_law():
    nU, nV, m = 400_000, 200_000, 8_000_000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.4, seed=11, device="cuda")
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    off, adj = oracle.build_csr(nU, nV, _np(eu), _np(ev))
    pairs = [(2, 2), (5, 3), (10, 10), (20, 5), (50, 50), (1, 100), (100, 1), (0, 30)]
    for mode in (-1, 0, 3):
        core.set_param("mode", mode)
        _check_pairs(core, nU, nV, eu, ev, pairs, off, adj)
    core.close()


def test_queue_knobs_keep_results_exact():
    # the cascade's work distribution (grab size, batch limits with and without the short limit
    # for a warp that drained the queue, chains of local batches, flush cadence) decides who walks
    # which row when, never the result
    nU, nV, m = 400_000, 200_000, 8_000_000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.4, seed=12, device="cuda")
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    off, adj = oracle.build_csr(nU, nV, _np(eu), _np(ev))
    want = {p: oracle.peel(nU, nV, off, adj, *p) for p in [(3, 3), (12, 6), (40, 40)]}
    knobs = [dict(batch_entries=128, batch_entries_small=0, local_rounds=0, grab_div=1, flush_steps=1),
             dict(batch_entries=4096, batch_entries_small=128, local_rounds=1, grab_div=0, flush_steps=16),
             dict(batch_entries=16384, batch_entries_small=512, local_rounds=256, grab_div=100000, flush_steps=4),
             dict(batch_entries=1024, batch_entries_small=4096, local_rounds=8, grab_div=64, flush_steps=4)]
    for kn in knobs:
        for k, v in kn.items():
            core.set_param(k, v)
        for round0 in (0, 1):
            core.set_param("round0", round0)
            for p, (wu, wv) in want.items():
                mu, mv = core.compute(*p)
                assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), (kn, round0, p)
    core.close()


def test_peel_full_size_4Mx2M_80M():
    """The five single peels at full size, each compared byte for byte with the oracle."""
    spec = synth.WORKLOADS["peel-4Mx2M-80M"]
    nU, nV, eu, ev = synth.make_graph(spec, device="cuda")
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    off, adj = oracle.build_csr(nU, nV, _np(eu), _np(ev))
    _check_pairs(core, nU, nV, eu, ev, spec["pairs"], off, adj)
    core.close()


def test_autotune_keeps_results_exact():
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
    pairs = [(2, 3), (3, 2), (5, 5), (8, 2)]
    best, chosen = core.autotune(pairs)
    assert best > 0
    assert chosen["blocks_per_sm"] in (0, 2, 3) and chosen["chunk"] in (256, 512, 1024, 2048)
    assert chosen["hub_degree"] in (0, 64, 256, 1024) and chosen["probe_bytes"] in (12, 16, 24, 32, 64)
    for a, b in pairs + [(1, 7), (4, 4)]:
        mu, mv = core.compute(a, b)
        wu, wv = oracle.peel(nU, nV, off, adj, a, b)
        assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv)
    best_b, chosen_b = core.autotune(synth.grid_pairs(4, 1, 8), batch=True)
    assert best_b > 0 and chosen_b["batch_wave"] in (2, 4, 8, 16)
    grid = synth.grid_pairs(4, 1, 8)
    bu, bv = core.compute_batch([p[0] for p in grid], [p[1] for p in grid])
    for i, (a, b) in enumerate(grid):
        wu, wv = oracle.peel(nU, nV, off, adj, a, b)
        assert np.array_equal(bu[i].cpu().numpy(), wu) and np.array_equal(bv[i].cpu().numpy(), wv)
    core.close()


def test_measure_atomics_reports_rates():
    core = ABCore(0)
    w, wo = core.measure_atomics(8 << 20)
    assert w > 1e9 and wo > 1e9  # at least a billion random atomics per second on any GB300
    with pytest.raises(ABCoreError):
        core.measure_atomics(16)
    core.close()


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_round0_first_round_without_returns(mode):
    # the initial candidate violators' rows walked by k_round0 (no-return decrements, then a scan
    # for what they took below the bound), in every mode with a searched layer, plain and pruned,
    # with every compiled walk (rows longer than 64 entries included: bounds up to 150)
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
    core.set_param("round0", 1)
    core.set_param("mode", mode)
    # (the last three leave a layer, or both, without candidates: empty hub tables)
    pairs = [(2, 3), (3, 2), (4, 4), (6, 2), (1, 9), (8, 8), (70, 3), (2, 150), (250, 2), (2, 250), (250, 250)]
    # variant 5 sums hub decrements in shared memory: no table, a table smaller than a warp, one
    # of a few rows' worth, and one larger than either candidate layer
    walks = [(v, 16384) for v in range(5)] + [(5, 0), (5, 7), (5, 64), (5, 16384)]
    sdecs = {}
    for variant, hub in walks:
        core.set_param("round0_variant", variant)
        core.set_param("round0_hub", hub)
        for a, b in pairs:
            core.set_param("reset_stats", 1)
            mu, mv = core.compute(a, b)
            st = core.stats()
            wu, wv = oracle.peel(nU, nV, off, adj, a, b)
            assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), (mode, variant, hub, a, b)
            # every walk makes the same decrements; only variant 5 with a table sums some of them
            assert sdecs.setdefault((a, b), st["stream_decrements"]) == st["stream_decrements"], (variant, hub, a, b)
            assert 0 <= st["hub_flushes"] <= st["hub_decrements"] <= st["stream_decrements"]
            if variant < 5 or hub == 0:
                assert st["hub_decrements"] == 0 and st["hub_flushes"] == 0
            elif hub == 16384 and mode == 3:
                # a table past both candidate layers holds every first-round target
                assert st["hub_decrements"] == st["stream_decrements"]
    core.set_param("round0_variant", 0)
    core.set_param("round0_hub", 16384)
    if mode == 3:
        core.core_numbers()
        core.set_param("algo", 2)
        for a, b in pairs:
            mu, mv = core.compute(a, b)
            wu, wv = oracle.peel(nU, nV, off, adj, a, b)
            assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), ("gcc+", a, b)
    core.close()


def _hub_graph(seed):
    # a few U hubs adjacent to most of V plus a sparse random part: long sorted rows whose
    # candidate boundary sits anywhere, including far from the layer-wide share
    rng = np.random.default_rng(seed)
    nU, nV = 3000, 2500
    hubs = 5
    eu = [np.full(nV - 100 * h, h) for h in range(hubs)]
    ev = [np.arange(100 * h, nV) for h in range(hubs)]
    m_rand = 30000
    eu.append(rng.integers(hubs, nU, m_rand))
    ev.append(rng.integers(0, nV, m_rand))
    eu, ev = np.concatenate(eu), np.concatenate(ev)
    key = np.unique(eu.astype(np.int64) * nV + ev)
    return nU, nV, (key // nV).astype(np.int32), (key % nV).astype(np.int32)


@pytest.mark.parametrize("seed", [0, 1])
def test_row_search_on_long_skewed_rows(seed):
    # every count by search (mode 3) over hub rows of 2000+ entries and short random rows, for
    # thresholds that move each layer's candidate boundary from a few ids to most of the layer
    nU, nV, eu, ev = _hub_graph(seed)
    off, adj = oracle.build_csr(nU, nV, eu, ev)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    core.set_param("mode", 3)
    for a, b in [(1, 1), (2, 2), (5, 1), (1, 6), (9, 3), (12, 12), (30, 2), (2, 40)]:
        mu, mv = core.compute(a, b)
        wu, wv = oracle.peel(nU, nV, off, adj, a, b)
        assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), (a, b)
    core.close()


@pytest.mark.parametrize("pdl", [0, 1])
def test_dependent_launches_back_to_back(pdl):
    # the kernels after the count init launched as programmatic dependents (or not): many
    # asynchronous peels in a row, in every counting mode and with round0, equal the oracle's
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    core.set_param("pdl", pdl)
    pairs = [(2, 3), (3, 2), (4, 4), (6, 2), (1, 9), (8, 8)]
    want = {p: oracle.peel(nU, nV, off, adj, *p) for p in pairs}
    for mode in (0, 1, 2, 3):
        for r0 in (0, 1):
            core.set_param("mode", mode)
            core.set_param("round0", r0)
            outs = []
            for a, b in pairs * 3:
                mu = torch.zeros(nU, dtype=torch.uint8, device="cuda")
                mv = torch.zeros(nV, dtype=torch.uint8, device="cuda")
                core.compute(a, b, mu, mv, asynchronous=True)
                outs.append(((a, b), mu, mv))
            core.sync()
            for p, mu, mv in outs:
                wu, wv = want[p]
                assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), (pdl, mode, r0, p)
    core.close()


def test_timing_kinds_selects_the_timed_launches():
    # events around the chosen kernel kinds only; the cores do not change
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    core.set_param("mode", 3)  # every count by search: init, then the cascade
    wu, wv = oracle.peel(nU, nV, off, adj, 3, 3)
    for kinds, timed in [(0xFF, (1, 0, 1)), (1 << abi.K_CASCADE, (0, 0, 1)), (1 << abi.K_INIT, (1, 0, 0))]:
        core.set_param("timing", 1)
        core.set_param("timing_kinds", kinds)
        core.set_param("reset_stats", 1)
        mu, mv = core.compute(3, 3)
        core.sync()
        st = core.stats()
        assert tuple(st["kernel_launches"][:3]) == timed, kinds
        assert (st["kernel_ms"][abi.K_CASCADE] > 0) == bool(timed[2])
        assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv)
    with pytest.raises(ABCoreError):
        core.set_param("timing_kinds", 256)
    core.close()


def test_round0_violator_list_longer_than_the_grid():
    # k_round0's grid is capped (16 blocks of 256 lanes per SM), so each warp walks several
    # groups of the violator list when it holds more entries than the grid has lanes; every
    # lane past the list's end must walk nothing. 4M x 4M vertices, 16M edges, light-tailed
    # degrees: (4,4) with every count by search leaves ~1.4M initial candidate violators.
    spec = dict(nU=4_000_000, nV=4_000_000, m=16_000_000, gamma_u=4.0, gamma_v=4.0, seed=7, kmax=None)
    nU, nV, eu, ev = synth.make_graph(spec)
    eu, ev = eu.numpy(), ev.numpy()
    off, adj = oracle.build_csr(nU, nV, eu, ev)
    lanes = torch.cuda.get_device_properties(0).multi_processor_count * 16 * 256
    deg = np.diff(off)
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    core.set_param("mode", 3)
    for a, b in [(4, 4), (3, 5), (3, 3)]:
        thr = np.concatenate([np.full(nU, a), np.full(nV, b)])
        cand = deg >= thr
        # live-candidate count of each candidate: its neighbours that are candidates
        csum = np.concatenate([[0], np.cumsum(cand[adj], dtype=np.int64)])
        nb_cand = csum[off[1:]] - csum[off[:-1]]
        n_viol = int((cand & (nb_cand < thr)).sum())
        if (a, b) == (4, 4):
            assert n_viol > 2 * lanes, (n_viol, lanes)  # several groups per warp
        wu, wv = oracle.peel(nU, nV, off, adj, a, b)
        for r0, variant in ((0, 0), (1, 0), (1, 4), (1, 5)):
            core.set_param("round0", r0)
            core.set_param("round0_variant", variant)
            mu, mv = core.compute(a, b)
            assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), (a, b, r0, variant)
    core.close()


@pytest.mark.parametrize("bitmap_pct", [0, 101])
def test_mask_gather_with_and_without_the_removal_bitmap(bitmap_pct):
    # the caller-order gather tests removal by bitmap (0: always) or by count (101: never), with
    # 4-byte mask stores (|U| a multiple of 4, masks aligned; |U| + |V| odd, so the last group
    # of four ids is partial) or byte stores (an odd |U|, or masks at odd offsets)
    for nU, nV, seed in [(4000, 2999, 13), (4001, 2999, 14)]:
        eu, ev = synth.chung_lu_edges(nU, nV, 40000, 2.2, 2.3, seed=seed)
        off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
        core = ABCore(0)
        core.load_edges(nU, nV, eu.cuda(), ev.cuda())
        core.set_param("emit_scatter_max_pct", 0)
        core.set_param("emit_bitmap_min_pct", bitmap_pct)
        for mode in (0, 3):
            core.set_param("mode", mode)
            for r0 in (0, 1):
                core.set_param("round0", r0)
                for a, b in [(1, 1), (2, 3), (4, 4), (7, 2), (12, 12), (0, 5)]:
                    wu, wv = oracle.peel(nU, nV, off, adj, a, b)
                    mu, mv = core.compute(a, b)
                    assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), (nU, mode, r0, a, b)
                    bu = torch.zeros(nU + 1, dtype=torch.uint8, device="cuda")
                    bv = torch.zeros(nV + 3, dtype=torch.uint8, device="cuda")
                    core.compute(a, b, bu[1:], bv[3:])
                    assert np.array_equal(bu[1:].cpu().numpy(), wu) and np.array_equal(bv[3:].cpu().numpy(), wv), ("unaligned", nU, a, b)
        core.close()


@pytest.mark.parametrize("swizzle", [0, 1])
def test_count_layouts_agree_with_the_oracle(swizzle):
    # counts in vertex order and in the swizzled layout (each layer's ids hashed over its
    # power-of-two range); layers whose sizes are and are not powers of two; single peels in every
    # counting mode with and without round0, and batch chains with 16- and 32-bit counts
    for nU, nV, m, seed in ((4096, 3000, 60_000, 3), (5000, 2048, 50_000, 4)):
        eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.3, seed=seed, kmax=300)
        eu, ev = eu.numpy(), ev.numpy()
        off, adj = oracle.build_csr(nU, nV, eu, ev)
        core = ABCore(0)
        core.set_param("count_swizzle", swizzle)
        core.load_edges(nU, nV, eu, ev)
        pairs = [(2, 3), (5, 5), (1, 12), (9, 2), (30, 30)]
        want = {p: oracle.peel(nU, nV, off, adj, *p) for p in pairs}
        for mode in (-1, 0, 3):
            for r0 in (0, 1):
                core.set_param("mode", mode)
                core.set_param("round0", r0)
                for p in pairs:
                    mu, mv = core.compute(*p)
                    assert np.array_equal(mu.cpu().numpy(), want[p][0]) and \
                        np.array_equal(mv.cpu().numpy(), want[p][1]), (swizzle, nU, mode, r0, p)
        core.set_param("mode", -1)
        grid = synth.grid_pairs(6, 1, 64)
        gw = {p: oracle.peel(nU, nV, off, adj, *p) for p in grid}
        for packed in (1, 0):
            core.set_param("packed_counts", packed)
            bu, bv = core.compute_batch([p[0] for p in grid], [p[1] for p in grid])
            bu, bv = bu.cpu().numpy(), bv.cpu().numpy()
            for i, p in enumerate(grid):
                assert np.array_equal(bu[i], gw[p][0]) and np.array_equal(bv[i], gw[p][1]), (swizzle, packed, p)
        core.close()


def test_log_level_2_queue_trace_keeps_results(capfd):
    # at log level 2 the cascade's watcher warp samples the queue instead of taking work and the
    # phase times are logged; the masks stay exact
    nU, nV, m = 400_000, 200_000, 8_000_000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.4, seed=13, device="cuda")
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    off, adj = oracle.build_csr(nU, nV, _np(eu), _np(ev))
    core.set_param("log_level", 2)
    for round0 in (0, 1):
        core.set_param("round0", round0)
        for a, b in [(3, 3), (25, 25)]:
            mu, mv = core.compute(a, b)
            wu, wv = oracle.peel(nU, nV, off, adj, a, b)
            assert np.array_equal(mu.cpu().numpy(), wu) and np.array_equal(mv.cpu().numpy(), wv), (round0, a, b)
    core.set_param("log_level", 0)
    core.close()
    err = capfd.readouterr().err
    assert "cascade queue drained after" in err and "cascade queue (time:done/tail/head)" in err


def test_mask_scatter_through_the_survivor_bitmap():
    # the scatter sets survivors' bits in a caller-order bitmap and k_expand writes every mask
    # byte from it: 16-byte stores where a word's 32 ids lie in one layer and the destination is
    # aligned, byte stores across the layer boundary, at odd offsets and in the last partial word;
    # stale bytes in the caller's buffers are overwritten, and the bitmap is clean for the next peel
    for nU, nV, seed in [(4000, 3008, 21), (4001, 2999, 22), (31, 5, 23)]:
        m = min(40000, nU * nV // 2)
        eu, ev = synth.chung_lu_edges(nU, nV, m, 2.2, 2.3, seed=seed)
        off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
        core = ABCore(0)
        core.load_edges(nU, nV, eu.cuda(), ev.cuda())
        core.set_param("emit_scatter_max_pct", 100)
        for r0 in (0, 1):
            core.set_param("round0", r0)
            for a, b in [(1, 1), (3, 2), (5, 5), (9, 2), (40, 40), (0, 0)]:
                wu, wv = oracle.peel(nU, nV, off, adj, a, b)
                for pad_u, pad_v in [(0, 0), (1, 3), (16, 7)]:
                    bu = torch.full((nU + pad_u,), 7, dtype=torch.uint8, device="cuda")
                    bv = torch.full((nV + pad_v,), 7, dtype=torch.uint8, device="cuda")
                    core.compute(a, b, bu[pad_u:], bv[pad_v:])
                    assert np.array_equal(bu[pad_u:].cpu().numpy(), wu), (nU, r0, a, b, pad_u)
                    assert np.array_equal(bv[pad_v:].cpu().numpy(), wv), (nV, r0, a, b, pad_v)
                    assert int(bu[:pad_u].ne(7).sum()) == 0 and int(bv[:pad_v].ne(7).sum()) == 0
        core.close()
