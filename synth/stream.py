"""Seeded edge-update streams for the on-the-fly query workload.

Op k of the stream, drawn with the counter-based hash (counter = k):

* insert with probability p_insert (default 0.7), else delete; a delete on an empty edge set
  becomes an insert;
* insert: u is the U endpoint of a uniformly chosen base edge and v the V endpoint of another
  (so both endpoints are degree-proportional); the pair is redrawn (attempt a = 1, 2, ...) until
  it is absent from the current edge set;
* delete: a uniform element of the current edge set, kept as an indexable array with swap-remove
  so that edges inserted earlier in the stream can be deleted too;
* target: uniform over the n_targets (alpha, beta) targets;
* arrival: unit-rate exponential inter-arrival times; the stream at rate lam uses times / lam, so
  the op sequence is the same at every rate.
"""

from dataclasses import dataclass

import numpy as np
import torch

from .rng import derive_key, uniform53

_ATTEMPTS = 16


@dataclass
class StreamOp:
    op: np.ndarray        # int8: 0 = insert, 1 = delete
    u: np.ndarray         # int32 U id
    v: np.ndarray         # int32 V id
    target: np.ndarray    # int8 index into the target list
    t_unit: np.ndarray    # float64 arrival time at unit rate (seconds * rate)

    def __len__(self):
        return len(self.op)


def _uniforms(n: int, seed: int, *purpose: int) -> np.ndarray:
    idx = torch.arange(n, dtype=torch.int64)
    return uniform53(idx, derive_key(seed, *purpose, 0), derive_key(seed, *purpose, 1)).numpy()


def edge_update_stream(eu: np.ndarray, ev: np.ndarray, nU: int, nV: int, n_ops: int, seed: int,
                       p_insert: float = 0.7, n_targets: int = 4) -> StreamOp:
    eu = np.asarray(eu, dtype=np.int64)
    ev = np.asarray(ev, dtype=np.int64)
    m = len(eu)
    base_sorted = np.sort(eu * nV + ev)

    def is_base(key):
        i = np.searchsorted(base_sorted, key)
        return i < m and base_sorted[i] == key

    r_op = _uniforms(n_ops, seed, 20)
    r_tg = _uniforms(n_ops, seed, 21)
    r_del = _uniforms(n_ops, seed, 22)
    r_arr = _uniforms(n_ops, seed, 23)
    r_ins = [(_uniforms(n_ops, seed, 24, a), _uniforms(n_ops, seed, 25, a)) for a in range(_ATTEMPTS)]

    cur = np.empty(m + n_ops, dtype=np.int64)
    cur[:m] = eu * nV + ev
    count = m
    inserted, deleted = set(), set()

    op = np.zeros(n_ops, dtype=np.int8)
    uu = np.zeros(n_ops, dtype=np.int32)
    vv = np.zeros(n_ops, dtype=np.int32)
    for k in range(n_ops):
        do_insert = r_op[k] < p_insert or count == 0
        if do_insert:
            if m == 0:
                raise ValueError("insert endpoints are drawn from base edges; base graph is empty")
            a = 0
            while True:
                if a < _ATTEMPTS:
                    r1, r2 = r_ins[a][0][k], r_ins[a][1][k]
                else:
                    idx = torch.tensor([k * 4096 + a], dtype=torch.int64)
                    r1 = float(uniform53(idx, derive_key(seed, 26, 0), derive_key(seed, 26, 1))[0])
                    r2 = float(uniform53(idx, derive_key(seed, 27, 0), derive_key(seed, 27, 1))[0])
                    if a > 100000:
                        raise RuntimeError("no absent pair found for an insert")
                u = int(eu[min(int(r1 * m), m - 1)])
                v = int(ev[min(int(r2 * m), m - 1)])
                key = u * nV + v
                base = is_base(key)
                present = (key in inserted) or (base and key not in deleted)
                if not present:
                    break
                a += 1
            if base:
                deleted.discard(key)
            else:
                inserted.add(key)
            cur[count] = key
            count += 1
            op[k] = 0
        else:
            i = min(int(r_del[k] * count), count - 1)
            key = int(cur[i])
            cur[i] = cur[count - 1]
            count -= 1
            if is_base(key):
                deleted.add(key)
            else:
                inserted.discard(key)
            u, v = key // nV, key % nV
            op[k] = 1
        uu[k] = u
        vv[k] = v
    target = np.minimum((r_tg * n_targets).astype(np.int64), n_targets - 1).astype(np.int8)
    t_unit = np.cumsum(-np.log1p(-r_arr))
    return StreamOp(op=op, u=uu, v=vv, target=target, t_unit=t_unit)


def sample_positions(stream: StreamOp, n_targets: int, per: int):
    """Update positions to check against a slow reference: for each kind of update and each
    target, `per` positions spread evenly over the stream, plus the first and the last update."""
    n = len(stream)
    ks = {0, n - 1} if n else set()
    for opk in (0, 1):
        for t in range(n_targets):
            idx = np.nonzero((stream.op == opk) & (stream.target == t))[0]
            if len(idx):
                ks.update(int(idx[j]) for j in np.linspace(0, len(idx) - 1, min(per, len(idx))).astype(np.int64))
    return sorted(ks)
