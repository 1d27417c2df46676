"""Cluster tree: Algs. 1-2, Appendix B and the array numbering of Section 8.

Test infrastructure only; see the package docstring.

Readings taken where the paper is silent or garbled:
* Depth (Section 8): all leaves sit at depth kappa = 0 if N <= N0 else
  ceil(log2(N/N0)), i.e. the smallest kappa with N0 * 2^kappa >= N.  The
  recursive rule of Alg. 2 ("split while |S| > N0") and this array rule agree
  whenever N/N0 is a power of two.
* Median (Alg. 2 line "k_split" is garbled; Appendix B is explicit): the
  first child S1 holds the ceil(|S|/2) members with the smallest coordinate
  along the split axis, the second child the rest.  Equal coordinates are
  ordered by original particle index, so membership is unique.
* Split axis (Alg. 1): argmax_k s_k (b_k - a_k) with s = (1, 1, gbar); on a
  tie the first axis in x, y, z order wins.
* Node numbering (Section 8): breadth first, root 1, children of i are 2i
  and 2i+1, level l holds nodes 2^l .. 2^(l+1)-1.
* Leaf size N0 >= 2, which with the balanced split keeps every node
  non-empty.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def tree_depth(N: int, N0: int) -> int:
    """kappa of Section 8: 0 if N <= N0, else the least k with N0 * 2^k >= N."""
    if N <= N0:
        return 0
    k = 0
    while N0 * (1 << k) < N:
        k += 1
    return k


def bbox(X: np.ndarray):
    """Bounding box of Section 2: a_g = min, b_g = max over the members."""
    return X.min(axis=0), X.max(axis=0)


def direction4split(lo: np.ndarray, hi: np.ndarray, s) -> int:
    """Alg. 1: argmax over k of s_k (b_k - a_k), first axis on ties."""
    w = [s[k] * (hi[k] - lo[k]) for k in range(3)]
    best = 0
    for k in (1, 2):
        if w[k] > w[best]:
            best = k
    return best


@dataclass
class Tree:
    N: int
    N0: int
    kappa: int
    gbar: float
    members: list          # members[i] = original indices of node i (index 0 unused)
    lo: np.ndarray         # [C+1, 3] lower box corners
    hi: np.ndarray         # [C+1, 3] upper box corners
    axis: np.ndarray       # [C+1] split axis of inner nodes, -1 at leaves

    @property
    def C(self) -> int:
        return (1 << (self.kappa + 1)) - 1

    def is_leaf(self, i: int) -> bool:
        return i >= (1 << self.kappa)

    def level(self, i: int) -> int:
        return i.bit_length() - 1

    def leaves(self):
        return range(1 << self.kappa, 1 << (self.kappa + 1))


def subdivide(x: np.ndarray, gbar: float, N0: int) -> Tree:
    """Alg. 2 applied from the root with the readings of the module docstring."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    if N0 < 2:
        raise ValueError("leaf size N0 must be >= 2")
    kappa = tree_depth(N, N0)
    C = (1 << (kappa + 1)) - 1
    s = (1.0, 1.0, gbar)
    members = [None] * (C + 1)
    lo = np.zeros((C + 1, 3))
    hi = np.zeros((C + 1, 3))
    axis = np.full(C + 1, -1, dtype=np.int64)

    def rec(i: int, idx: np.ndarray, level: int):
        members[i] = idx
        lo[i], hi[i] = bbox(x[idx])
        if level == kappa:
            return
        k = direction4split(lo[i], hi[i], s)
        axis[i] = k
        order = np.lexsort((idx, x[idx, k]))  # primary: coordinate, secondary: index
        h1 = (idx.size + 1) // 2
        rec(2 * i, idx[order[:h1]], level + 1)
        rec(2 * i + 1, idx[order[h1:]], level + 1)

    rec(1, np.arange(N, dtype=np.int64), 0)
    return Tree(N, N0, kappa, gbar, members, lo, hi, axis)
