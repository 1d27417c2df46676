"""Pins of the oracle's interpolation basis (Section 2, Theorem 1) on the CPU."""
import numpy as np
import pytest
import torch
from numpy.polynomial import chebyshev as C
from scipy.interpolate import BarycentricInterpolator

from oracle import interp


@pytest.mark.parametrize("n", [1, 2, 4, 7, 10, 12])
def test_points_are_chebyshev_extrema(n):
    t = interp.cheb_points(n)
    assert t[0] == 1.0 and t[-1] == -1.0 and np.all(np.diff(t) < 0)
    Tn = C.Chebyshev.basis(n)
    np.testing.assert_allclose(Tn(t), (-1.0) ** np.arange(n + 1), atol=1e-12)


@pytest.mark.parametrize("n", [1, 3, 4, 6, 8, 12])
def test_basis_cardinal_partition_and_scipy(n):
    a, b = -0.3, 1.9
    xi = interp.points_1d(a, b, n)
    L = interp.lagrange_1d(torch.as_tensor(xi), a, b, n).numpy()
    np.testing.assert_allclose(L, np.eye(n + 1), atol=1e-12)
    x = np.linspace(a - 0.1, b + 0.1, 57)
    L = interp.lagrange_1d(torch.as_tensor(x), a, b, n).numpy()
    np.testing.assert_allclose(L.sum(1), 1.0, atol=1e-12)
    # against scipy's barycentric interpolator on the same points
    for k in range(n + 1):
        e = np.zeros(n + 1)
        e[k] = 1.0
        ref = BarycentricInterpolator(xi, e)(x)
        np.testing.assert_allclose(L[:, k], ref, atol=1e-11)


@pytest.mark.parametrize("n", [2, 5, 9])
def test_theorem1_polynomial_reproduction(n):
    """Theorem 1: sum_k P(xi_k) l_k(x) = P(x) for deg P <= n, and not for deg n+1."""
    a, b = 1.0, 4.0
    rng = np.random.default_rng(n)
    coef = rng.standard_normal(n + 1)
    xi = interp.points_1d(a, b, n)
    x = rng.uniform(a, b, 40)
    L = interp.lagrange_1d(torch.as_tensor(x), a, b, n).numpy()
    np.testing.assert_allclose(L @ np.polyval(coef, xi), np.polyval(coef, x), rtol=1e-10, atol=1e-10)
    coef2 = np.concatenate([[1.0], coef])
    assert np.abs(L @ np.polyval(coef2, xi) - np.polyval(coef2, x)).max() > 1e-6


def test_degenerate_side_and_3d_layout():
    L = interp.lagrange_1d(torch.tensor([2.5, 2.5]), 2.5, 2.5, 4).numpy()
    np.testing.assert_array_equal(L, [[1, 0, 0, 0, 0]] * 2)
    lo, hi, n = np.array([0.0, 1.0, 2.0]), np.array([1.0, 3.0, 2.0]), 3
    P = interp.proxy_points(lo, hi, n)
    assert P.shape == (64, 3)
    # x fastest: nu = nu1 + 4 nu2 + 16 nu3
    np.testing.assert_allclose(P[1], [interp.points_1d(0, 1, 3)[1], interp.points_1d(1, 3, 3)[0], 2.0])
    np.testing.assert_allclose(P[4], [interp.points_1d(0, 1, 3)[0], interp.points_1d(1, 3, 3)[1], 2.0])
    B = interp.basis_3d(torch.as_tensor(P), lo, hi, n).numpy()
    # the z side is degenerate: every point collapses onto the nu3 = 0 layer
    np.testing.assert_allclose(B[:16, :16], np.eye(16), atol=1e-12)
    np.testing.assert_allclose(B.sum(1), 1.0, atol=1e-12)
