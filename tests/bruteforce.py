"""Independent checks used to pin the oracle: subset enumeration and fixture parsing.

Nothing here peels. ``max_feasible`` enumerates every vertex subset of a tiny graph, keeps the
ones that meet Definition 1's degree bounds inside themselves, and returns their union, which
must itself be feasible (so it is the unique maximal one).
"""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def nbr_masks(nU, nV, edges):
    n = nU + nV
    nb = [0] * n
    for u, v in edges:
        x, y = u, nU + v
        nb[x] |= 1 << y
        nb[y] |= 1 << x
    return nb


def feasible(S, nU, nb, alpha, beta):
    x = 0
    T = S
    while T:
        if T & 1:
            thr = alpha if x < nU else beta
            if bin(nb[x] & S).count("1") < thr:
                return False
        T >>= 1
        x += 1
    return True


def max_feasible(nU, nV, edges, alpha, beta):
    """Union of all feasible vertex subsets (as a bitmask), asserting the union is feasible."""
    n = nU + nV
    assert n <= 16
    nb = nbr_masks(nU, nV, edges)
    union = 0
    for S in range(1 << n):
        if S & ~union == 0:
            continue  # adds nothing new to the union
        if feasible(S, nU, nb, alpha, beta):
            union |= S
    assert feasible(union, nU, nb, alpha, beta), "union of feasible subsets must be feasible"
    return union


def mask_from_bits(bits, nU, nV):
    mu = np.array([(bits >> u) & 1 for u in range(nU)], dtype=np.uint8)
    mv = np.array([(bits >> (nU + v)) & 1 for v in range(nV)], dtype=np.uint8)
    return mu, mv


def load_paper_examples():
    """Parse tests/golden/paper_examples.txt into a list of steps."""
    path = os.path.join(GOLDEN, "paper_examples.txt")
    graph = None
    edges = []
    steps = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "graph":
                graph = (int(tok[1]), int(tok[2]))
            elif tok[0] == "edge":
                edges.append((int(tok[1]), int(tok[2])))
            elif tok[0] == "core":
                _, a, b, rest = line.split(None, 3)
                parts = rest.split("|")
                us = [int(t) for t in parts[1].split()]
                vs = [int(t) for t in parts[2].split()]
                steps.append(("core", int(a), int(b), us, vs))
            elif tok[0] == "corenum":
                steps.append(("corenum", [int(t) for t in tok[1:]]))
            elif tok[0] == "insert":
                steps.append(("insert", int(tok[1]), int(tok[2])))
    return graph, edges, steps
