"""GPU parity of the batched cores (nested chains, one persistent launch, CUDA-graph replay).

Every pair's masks must equal the oracle's peel of that pair on the full graph, and equal the
plain single peel, whatever the order of the pair list."""

import random

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2606_07148_gb300 import ABCore

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_07148_gb300.buildlib import build
    build()


def _check_batch(core, nU, nV, off, adj, pairs, out=None):
    a = [p[0] for p in pairs]
    b = [p[1] for p in pairs]
    mu, mv = core.compute_batch(a, b) if out is None else core.compute_batch(a, b, *out)
    mu = mu.cpu().numpy() if isinstance(mu, torch.Tensor) else mu
    mv = mv.cpu().numpy() if isinstance(mv, torch.Tensor) else mv
    cache = {}
    for i, (x, y) in enumerate(pairs):
        if (x, y) not in cache:
            cache[(x, y)] = oracle.peel(nU, nV, off, adj, x, y)
        wu, wv = cache[(x, y)]
        assert np.array_equal(mu[i], wu) and np.array_equal(mv[i], wv), \
            "pair %d (%d,%d): U diff %d V diff %d" % (i, x, y, int((mu[i] != wu).sum()), int((mv[i] != wv).sum()))
    return mu, mv


@pytest.fixture(scope="module")
def small():
    nU, nV, eu, ev = synth.make_graph("peel-2000x1500-20k")
    off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
    return nU, nV, eu, ev, off, adj


def test_batch_grid_16x16_small_graph(small):
    nU, nV, eu, ev, off, adj = small
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    pairs = synth.grid_pairs(16, 1, 512)
    _check_batch(core, nU, nV, off, adj, pairs)
    # replay of the captured graph, same outputs
    mu, mv = core.compute_batch([p[0] for p in pairs], [p[1] for p in pairs])
    mu2, mv2 = core.compute_batch([p[0] for p in pairs], [p[1] for p in pairs], mu.clone(), mv.clone())
    assert torch.equal(mu, mu2) and torch.equal(mv, mv2)
    core.close()


@pytest.mark.parametrize("mode", [-1, 0, 3])
def test_batch_shuffled_pairs_with_duplicates_and_zeros(small, mode):
    nU, nV, eu, ev, off, adj = small
    rng = random.Random(5 + mode)
    core = ABCore(0)
    core.set_param("mode", mode)
    core.set_param("chunk", 64)
    core.load_edges(nU, nV, eu.numpy(), ev.numpy())
    vals = [0, 1, 2, 3, 4, 6, 9, 15, 40, 300]
    pairs = [(rng.choice(vals), rng.choice(vals)) for _ in range(70)]
    pairs += [pairs[3], pairs[7], (0, 0), (2, 0), (0, 2)]
    rng.shuffle(pairs)
    _check_batch(core, nU, nV, off, adj, pairs)
    core.close()


def test_batch_equals_plain_peels_and_host_pointers(small):
    nU, nV, eu, ev, off, adj = small
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    pairs = synth.grid_pairs(8, 1, 1024)
    hu = np.zeros((len(pairs), nU), np.uint8)
    hv = np.zeros((len(pairs), nV), np.uint8)
    _check_batch(core, nU, nV, off, adj, pairs, out=(hu, hv))
    for i, (a, b) in enumerate(pairs):
        mu, mv = core.compute(a, b)
        assert np.array_equal(mu.cpu().numpy(), hu[i]) and np.array_equal(mv.cpu().numpy(), hv[i])
    core.close()


def test_batch_tiny_random_graphs():
    rng = random.Random(23)
    core = ABCore(0)
    for _ in range(15):
        nU, nV = rng.randint(1, 14), rng.randint(1, 14)
        edges = [(u, v) for u in range(nU) for v in range(nV) if rng.random() < rng.uniform(0.1, 0.9)]
        eu = np.array([e[0] for e in edges], dtype=np.int32)
        ev = np.array([e[1] for e in edges], dtype=np.int32)
        core.load_edges(nU, nV, eu, ev)
        off, adj = oracle.build_csr(nU, nV, eu, ev)
        pairs = [(rng.randint(0, 6), rng.randint(0, 6)) for _ in range(20)]
        _check_batch(core, nU, nV, off, adj, pairs)
    core.close()


def test_batch_mid_size_power_law():
    nU, nV, m = 400_000, 200_000, 8_000_000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.2, seed=12, device="cuda")
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    off, adj = oracle.build_csr(nU, nV, eu.cpu().numpy(), ev.cpu().numpy())
    pairs = synth.grid_pairs(8, 1, 1024)
    _check_batch(core, nU, nV, off, adj, pairs)
    core.close()


def test_batch_with_32_bit_counts(small):
    # the chains keep 16-bit counts whenever every degree fits; the 32-bit path must agree
    nU, nV, eu, ev, off, adj = small
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    pairs = synth.grid_pairs(8, 1, 64)
    mu16, mv16 = _check_batch(core, nU, nV, off, adj, pairs)
    core.set_param("packed_counts", 0)
    assert core.get_param("packed_counts") == 0
    mu32, mv32 = _check_batch(core, nU, nV, off, adj, pairs)
    assert np.array_equal(mu16, mu32) and np.array_equal(mv16, mv32)
    core.close()


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("wave", [1, 3])
def test_batch_seeding_and_waves(small, seed, wave):
    # with and without seeding from the finished chain of a smaller alpha; one chain per wave
    # (every chain but the first seeded) and three (chains of the first wave unseeded)
    nU, nV, eu, ev, off, adj = small
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    core.set_param("batch_seed", seed)
    core.set_param("batch_wave", wave)
    pairs = synth.grid_pairs(8, 1, 64)
    _check_batch(core, nU, nV, off, adj, pairs)
    # the same list twice: the replay starts from a cleared record
    _check_batch(core, nU, nV, off, adj, pairs)
    core.close()


def test_batch_more_chains_than_own_record_columns(small):
    # beyond 64 distinct alphas the chains share record columns by wave slot (no seeding)
    nU, nV, eu, ev, off, adj = small
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    core.set_param("batch_seed", 1)
    pairs = [(a, b) for a in range(1, 71) for b in (1, 3, 9)]
    _check_batch(core, nU, nV, off, adj, pairs)
    core.close()


def test_batch_deep_beta_ladders_mid_size_power_law():
    # deep beta ladders on a skewed graph: every step moves U rows' boundaries across many V ids
    nU, nV, m = 400_000, 200_000, 8_000_000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.0, 2.3, seed=14, device="cuda")
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    off, adj = oracle.build_csr(nU, nV, eu.cpu().numpy(), ev.cpu().numpy())
    pairs = synth.grid_pairs(8, 1, 1024) + [(2, b) for b in range(2, 60, 3)]
    for seed in (0, 1):
        core.set_param("batch_seed", seed)
        _check_batch(core, nU, nV, off, adj, pairs)
    core.close()


@pytest.mark.parametrize("below", [0, 4, 1 << 30])
def test_batch_small_alphas_left_to_single_peels(small, below):
    # pairs with alpha below the split are computed by the single plain peel into their rows, the
    # rest by chains; every pair equals the oracle's, whatever the split (all chains, some, none)
    nU, nV, eu, ev, off, adj = small
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    core.core_numbers()  # prepared core numbers must not leak the pruned peel into the batch
    core.set_param("batch_plain_below", below)
    pairs = synth.grid_pairs(8, 1, 64) + [(0, 5), (5, 0)]
    _check_batch(core, nU, nV, off, adj, pairs)
    _check_batch(core, nU, nV, off, adj, pairs)
    core.close()


@pytest.mark.parametrize("nU, nV", [(4000, 3000), (4001, 2999), (4002, 3002)])
def test_batch_emit_widths(nU, nV):
    # the masks are written four caller ids at a time when both layers' sizes are multiples of
    # four (and the wave's removal steps fit one 4-byte row), else one id at a time
    eu, ev = synth.chung_lu_edges(nU, nV, 40_000, 2.2, 2.3, seed=nU + nV)
    off, adj = oracle.build_csr(nU, nV, eu.numpy(), ev.numpy())
    core = ABCore(0)
    core.load_edges(nU, nV, eu.cuda(), ev.cuda())
    _check_batch(core, nU, nV, off, adj, synth.grid_pairs(5, 1, 40))
    core.close()


@pytest.mark.parametrize("per_sm", [2, 3])
def test_batch_kernel_occupancies(per_sm):
    # the batch kernel is compiled for two and for three blocks an SM; both give the same masks
    nU, nV, m = 400_000, 200_000, 8_000_000
    eu, ev = synth.chung_lu_edges(nU, nV, m, 2.1, 2.2, seed=15, device="cuda")
    core = ABCore(0)
    core.load_edges(nU, nV, eu, ev)
    off, adj = oracle.build_csr(nU, nV, eu.cpu().numpy(), ev.cpu().numpy())
    core.set_param("blocks_per_sm", per_sm)
    _check_batch(core, nU, nV, off, adj, synth.grid_pairs(6, 1, 512))
    core.close()
