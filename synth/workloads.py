"""Named synthetic workloads, by what they are and their sizes.

Each entry fixes the Chung-Lu parameters (vertex counts, edge count, power-law exponents, seed,
kmax) plus the (alpha, beta) queries run on it. The paper's KONECT graphs and its synthetic PL
graph are not available here; these stand in for them.
"""

from .chung_lu import chung_lu_edges
from .grids import grid_pairs

WORKLOADS = {
    # small plain peel: seed 0, 2000 x 1500, 20k edges, exponent 2.3 on both layers, degrees <= 200
    "peel-2000x1500-20k": dict(nU=2000, nV=1500, m=20000, gamma_u=2.3, gamma_v=2.3, seed=0,
                               kmax=200, pairs=[(2, 3)]),
    # plain single peels: seed 1, 4M x 2M, 80M edges, exponents 2.1 / 2.4
    "peel-4Mx2M-80M": dict(nU=4_000_000, nV=2_000_000, m=80_000_000, gamma_u=2.1, gamma_v=2.4,
                           seed=1, kmax=None,
                           pairs=[(2, 2), (5, 3), (10, 10), (20, 5), (50, 50)]),
    # batched cores: seed 2, 20M x 10M, 500M edges, exponents 2.1 / 2.2, 16 x 16 grid in [1, 512]
    "batch-20Mx10M-500M": dict(nU=20_000_000, nV=10_000_000, m=500_000_000, gamma_u=2.1,
                               gamma_v=2.2, seed=2, kmax=None, pairs=grid_pairs(16, 1, 512)),
    # billion scale: seed 3, 100M x 50M, 1.5B edges, exponents 2.0 / 2.3,
    # one (64, 64) core plus an 8 x 8 grid in [1, 1024]
    "billion-100Mx50M-1500M": dict(nU=100_000_000, nV=50_000_000, m=1_500_000_000, gamma_u=2.0,
                                   gamma_v=2.3, seed=3, kmax=None,
                                   pairs=[(64, 64)] + grid_pairs(8, 1, 1024)),
    # the billion-scale recipe at a fifth of the vertices and a fifth of the edges (2.6 GB of
    # CSR): small enough for a profiler that replays each launch many times, with the counts of
    # a (64, 64) query still far beyond the L2
    "profile-20Mx10M-300M": dict(nU=20_000_000, nV=10_000_000, m=300_000_000, gamma_u=2.0,
                                 gamma_v=2.3, seed=3, kmax=None, pairs=[(64, 64)]),
    # the batch recipe at a fifth of the vertices and of the edges (0.85 GB of CSR, 1.5 GB of
    # masks): small enough for a profiler that replays each launch many times
    "batch-4Mx2M-100M": dict(nU=4_000_000, nV=2_000_000, m=100_000_000, gamma_u=2.1, gamma_v=2.2,
                             seed=2, kmax=None, pairs=grid_pairs(16, 1, 512)),
    # serving: seed 4, 10M x 5M, 200M edges, exponents 2.1 / 2.2, 100k updates
    "serve-10Mx5M-200M": dict(nU=10_000_000, nV=5_000_000, m=200_000_000, gamma_u=2.1,
                              gamma_v=2.2, seed=4, kmax=None, n_ops=100_000,
                              rates=[5_000, 20_000, 80_000],
                              targets=[(2, 2), (5, 5), (10, 20), (32, 32)]),
    # the serving recipe scaled down so the oracle can replay the whole stream
    "serve-10kx5k-200k": dict(nU=10_000, nV=5_000, m=200_000, gamma_u=2.1, gamma_v=2.2, seed=4,
                              kmax=None, n_ops=100_000, rates=[5_000, 20_000, 80_000],
                              targets=[(2, 2), (5, 5), (10, 20), (32, 32)]),
}


def make_graph(name_or_spec, device="cpu"):
    """(nU, nV, eu, ev) for a named workload (or a dict with the same keys)."""
    spec = WORKLOADS[name_or_spec] if isinstance(name_or_spec, str) else name_or_spec
    eu, ev = chung_lu_edges(spec["nU"], spec["nV"], spec["m"], spec["gamma_u"], spec["gamma_v"],
                            spec["seed"], kmax=spec.get("kmax"), device=device)
    return spec["nU"], spec["nV"], eu, ev
