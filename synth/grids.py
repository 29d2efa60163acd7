"""Log-spaced (alpha, beta) grids.

A grid of k values in [lo, hi] takes lo * (hi/lo)^(i/(k-1)), rounds half up, and bumps any value
that does not exceed its predecessor to predecessor + 1, so the sequence is strictly increasing.
With 16 values in [1, 512] this gives 1 2 3 4 5 8 12 18 28 42 64 97 147 223 338 512; with 8
values in [1, 1024] it gives 1 3 7 20 53 141 380 1024. Pairs are the Cartesian product, listed
alpha-major.
"""

import math


def log_grid(k: int, lo: int, hi: int):
    if k == 1:
        return [lo]
    out = []
    for i in range(k):
        x = lo * (hi / lo) ** (i / (k - 1))
        r = int(math.floor(x + 0.5))
        if out and r <= out[-1]:
            r = out[-1] + 1
        out.append(r)
    return out


def grid_pairs(k: int, lo: int, hi: int):
    g = log_grid(k, lo, hi)
    return [(a, b) for a in g for b in g]
