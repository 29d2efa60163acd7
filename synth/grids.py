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


def sampled_pairs(grid, limit):
    """Pairs of a grid to check against a slow reference: the four corners first, then the first
    and last beta of each alpha's chain, then the diagonal, up to `limit` distinct pairs."""
    al = sorted({p[0] for p in grid})
    be = sorted({p[1] for p in grid})
    order = [(al[0], be[0]), (al[0], be[-1]), (al[-1], be[0]), (al[-1], be[-1])]
    for a in al[1:-1]:
        order += [(a, be[-1]), (a, be[0])]
    order += [(a, b) for a, b in zip(al, be)]
    gs = set(map(tuple, grid))
    out = []
    for p in order:
        if p in gs and p not in out:
            out.append(p)
    return out[:limit]
