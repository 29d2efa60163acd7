"""Seeded synthetic inputs for the (alpha, beta)-core library, its tests and its benchmark.

This package holds input generation only -- random bipartite graphs (Chung-Lu), edge-update
streams with Poisson arrivals, and the log-spaced (alpha, beta) grids. It contains none of the
core arithmetic, so both the CUDA path and the CPU oracle may take their inputs from it without
sharing any of the method's code.
"""

from .rng import mix32, uniform53, derive_key
from .chung_lu import layer_weights, chung_lu_edges
from .stream import edge_update_stream, StreamOp, sample_positions
from .grids import log_grid, grid_pairs, sampled_pairs
from .workloads import WORKLOADS, make_graph

__all__ = [
    "mix32", "uniform53", "derive_key",
    "layer_weights", "chung_lu_edges",
    "edge_update_stream", "StreamOp", "sample_positions",
    "log_grid", "grid_pairs", "sampled_pairs",
    "WORKLOADS", "make_graph",
]
