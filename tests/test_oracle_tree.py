"""Pins of the oracle's cluster tree (Algs. 1-2, Appendix B, Section 8) on the CPU."""
import math

import numpy as np
import pytest

from oracle import tree as T
from paper_2302_07567_gb300.workloads import random_beam


@pytest.mark.parametrize("N,N0,k", [(1, 2, 0), (64, 64, 0), (65, 64, 1), (128, 64, 1), (129, 64, 2),
                                    (4096, 64, 6), (65536, 128, 9), (1 << 24, 256, 16), (3, 2, 1)])
def test_depth(N, N0, k):
    assert T.tree_depth(N, N0) == k
    if N > N0:
        assert k == math.ceil(math.log2(N / N0))


def _check_tree(x, tr):
    N = x.shape[0]
    assert sorted(tr.members[1].tolist()) == list(range(N))
    s = (1.0, 1.0, tr.gbar)
    for i in range(1, tr.C + 1):
        idx = tr.members[i]
        assert idx.size >= 1
        np.testing.assert_array_equal(tr.lo[i], x[idx].min(0))
        np.testing.assert_array_equal(tr.hi[i], x[idx].max(0))
        if tr.is_leaf(i):
            assert idx.size <= tr.N0
            continue
        L, R = tr.members[2 * i], tr.members[2 * i + 1]
        assert L.size == (idx.size + 1) // 2 and L.size + R.size == idx.size
        assert sorted(np.concatenate([L, R]).tolist()) == sorted(idx.tolist())
        k = tr.axis[i]
        w = [s[d] * (tr.hi[i][d] - tr.lo[i][d]) for d in range(3)]
        assert w[k] == max(w) and all(w[d] < w[k] for d in range(k))
        # every left member precedes every right member in (coordinate, index) order
        lmax = max(zip(x[L, k], L))
        rmin = min(zip(x[R, k], R))
        assert lmax < rmin


@pytest.mark.parametrize("N,N0", [(1000, 16), (4096, 64), (777, 5), (5, 2)])
def test_tree_structure(N, N0):
    x, p, q = random_beam(N, seed=N)
    tr = T.subdivide(x, 7.0, N0)
    assert tr.kappa == T.tree_depth(N, N0)
    _check_tree(x, tr)
    sizes = [tr.members[i].size for i in tr.leaves()]
    assert max(sizes) - min(sizes) <= 1


def test_ties_split_by_original_index():
    """Integer coordinates with many ties: membership is fixed by the index order."""
    rng = np.random.default_rng(0)
    x = rng.integers(0, 3, size=(300, 3)).astype(np.float64)
    tr = T.subdivide(x, 1.0, 8)
    _check_tree(x, tr)
    # root split: axis 0 (all widths equal to 2, first axis wins); the 150
    # smallest by (x, index) form the first child
    assert tr.axis[1] == 0
    order = sorted(range(300), key=lambda j: (x[j, 0], j))
    assert sorted(tr.members[2].tolist()) == sorted(order[:150])


def test_stretch_changes_split_axis():
    x = np.zeros((64, 3))
    x[:, 0] = np.linspace(0, 1.0, 64)
    x[:, 2] = np.linspace(0, 0.1, 64)[::-1]
    assert T.subdivide(x, 1.0, 8).axis[1] == 0
    assert T.subdivide(x, 20.0, 8).axis[1] == 2     # gbar * 0.1 > 1
