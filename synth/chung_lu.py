"""Seeded Chung-Lu bipartite graphs with power-law expected degrees.

Recipe (identical on CPU and GPU):

* Layer X with n_X vertices and exponent gamma_X gets rank weights w_i = (i+1)^(-1/(gamma_X-1)),
  scaled so that sum(w) = m, clipped to [kmin, kmax] and the unclipped part rescaled (at most 20
  rounds) so the sum stays m. kmax defaults to floor(sqrt(m)), which keeps every
  w_u * w_v / m <= 1.
* The U ranks are cut into buckets of about equal weight (one bucket per 2^26 edges). Bucket b
  receives m_b edges, its weight share of m rounded by largest remainder, so that sum m_b = m.
* Inside bucket b, draw t (a 64-bit counter) picks a U rank from the bucket's weights and a V rank
  from all V weights, both by inverse CDF over float64 prefix sums, with uniforms from the
  counter-based hash in ``synth.rng``. Repeated (u, v) keys are dropped (the first draw wins) and
  the bucket draws more until it holds exactly m_b distinct edges. U ranges of different buckets
  are disjoint, so no edge can repeat across buckets.
* Ranks become vertex ids through a seeded random permutation per layer, so the hubs do not sit
  at the low ids.

Edges come out bucket by bucket, each bucket in draw order.
"""

import math

import numpy as np
import torch

from .rng import M32, derive_key, mix32, uniform53

BUCKET_EDGES = 1 << 26


def layer_weights(n: int, gamma: float, m: int, kmin: float = 1.0, kmax: float = None) -> np.ndarray:
    """Expected degrees of one layer in rank order (non-increasing), summing to m."""
    if kmax is None:
        kmax = float(math.isqrt(m))
    i = np.arange(n, dtype=np.float64)
    w = (i + 1.0) ** (-1.0 / (gamma - 1.0))
    w *= m / w.sum()
    for _ in range(20):
        w = np.clip(w, kmin, kmax)
        free = (w > kmin) & (w < kmax)
        if not free.any():
            break
        fixed = w[~free].sum()
        scale = (m - fixed) / w[free].sum()
        if abs(scale - 1.0) < 1e-13:
            break
        w[free] *= scale
    return w


def _permutation(n: int, key: int, device) -> torch.Tensor:
    """perm[r] = vertex id given to rank r (a seeded random permutation)."""
    i = torch.arange(n, dtype=torch.int64, device=device)
    h1 = mix32(mix32((i & M32) ^ key) ^ (i >> 32))
    h2 = mix32(h1 ^ (key ^ 0x5BD1E995))
    h = (h1 << 31) | (h2 >> 1)
    return torch.sort(h, stable=True).indices


def _first_distinct(keys: torch.Tensor) -> torch.Tensor:
    """Mask of the first occurrence of every key, keys given in draw order."""
    sk, order = torch.sort(keys, stable=True)
    first = torch.ones_like(sk, dtype=torch.bool)
    if sk.numel() > 1:
        first[1:] = sk[1:] != sk[:-1]
    mask = torch.zeros_like(first)
    mask[order[first]] = True
    return mask


def _largest_remainder(total: int, shares: np.ndarray) -> np.ndarray:
    raw = shares / shares.sum() * total
    base = np.floor(raw).astype(np.int64)
    rest = int(total - base.sum())
    if rest > 0:
        frac = raw - base
        order = np.lexsort((np.arange(len(frac)), -frac))
        base[order[:rest]] += 1
    return base


def chung_lu_edges(nU: int, nV: int, m: int, gamma_u: float, gamma_v: float, seed: int,
                   kmax: float = None, kmin: float = 1.0, device="cpu",
                   bucket_edges: int = BUCKET_EDGES):
    """Return (eu, ev): int32 tensors of m distinct edges (per-layer vertex ids) on ``device``."""
    if m <= 0:
        z = torch.zeros(0, dtype=torch.int32, device=device)
        return z, z.clone()
    if m > nU * nV:
        raise ValueError("more edges requested than vertex pairs exist")
    wU = layer_weights(nU, gamma_u, m, kmin, kmax)
    wV = layer_weights(nV, gamma_v, m, kmin, kmax)
    cU_np = np.cumsum(wU)
    cV_np = np.cumsum(wV)
    cU = torch.from_numpy(cU_np).to(device)
    cV = torch.from_numpy(cV_np).to(device)
    totV = float(cV_np[-1])

    nb = max(1, -(-m // bucket_edges))
    tot = float(cU_np[-1])
    cuts = [0]
    for j in range(1, nb):
        c = int(np.searchsorted(cU_np, tot * j / nb, side="right"))
        if cuts[-1] < c < nU:
            cuts.append(c)
    cuts.append(nU)
    lo = np.array(cuts[:-1], dtype=np.int64)
    hi = np.array(cuts[1:], dtype=np.int64)
    wb = cU_np[hi - 1] - np.where(lo > 0, cU_np[np.maximum(lo - 1, 0)], 0.0)
    mb = _largest_remainder(m, wb)

    parts_u, parts_v = [], []
    for b in range(len(lo)):
        need_total = int(mb[b])
        if need_total == 0:
            continue
        blo, bhi = int(lo[b]), int(hi[b])
        if need_total > (bhi - blo) * nV:
            raise ValueError("bucket cannot hold its share of distinct edges")
        base = float(cU_np[blo - 1]) if blo > 0 else 0.0
        width = float(wb[b])
        ku = (derive_key(seed, 1, b, 0), derive_key(seed, 1, b, 1))
        kv = (derive_key(seed, 2, b, 0), derive_key(seed, 2, b, 1))
        acc = torch.zeros(0, dtype=torch.int64, device=device)
        drawn = 0
        stall = 0
        while acc.numel() < need_total:
            need = need_total - acc.numel()
            cnt = need + need // 8 + 64
            idx = torch.arange(drawn, drawn + cnt, dtype=torch.int64, device=device)
            drawn += cnt
            ru = uniform53(idx, *ku)
            rank_u = torch.searchsorted(cU, base + ru * width, right=True).clamp_(blo, bhi - 1)
            rv = uniform53(idx, *kv)
            rank_v = torch.searchsorted(cV, rv * totV, right=True).clamp_(0, nV - 1)
            del idx, ru, rv
            keys = rank_u * nV + rank_v
            del rank_u, rank_v
            allk = torch.cat([acc, keys])
            before = acc.numel()
            acc = allk[_first_distinct(allk)]
            del allk, keys
            stall = stall + 1 if acc.numel() == before else 0
            if stall > 64:
                raise RuntimeError("Chung-Lu draw made no progress; graph too dense for its weights")
        acc = acc[:need_total]
        parts_u.append(acc // nV)
        parts_v.append(acc % nV)
        del acc
    ranks_u = torch.cat(parts_u)
    ranks_v = torch.cat(parts_v)
    permU = _permutation(nU, derive_key(seed, 3), device)
    permV = _permutation(nV, derive_key(seed, 4), device)
    eu = permU[ranks_u].to(torch.int32)
    ev = permV[ranks_v].to(torch.int32)
    return eu, ev
