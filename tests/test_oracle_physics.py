"""Pins of the oracle's kernel and direct sums against closed forms (CPU).

Each test checks the oracle against physics or mathematics fixed outside it:
the field of a uniformly moving point charge (textbook form in terms of the
angle between R and the velocity), Coulomb's law for a symmetric
configuration, the Lorentz transformation of a rest-frame Coulomb field,
momentum conservation and invariances.
"""
import math

import numpy as np
import pytest

from oracle import bldtt, physics
from oracle.physics import C0, KE
from paper_2302_07567_gb300.workloads import random_beam


def _moving_charge_field(q, gamma, R):
    """Field at R (from the charge's present position) of a charge moving along z.

    Textbook form: E = q (1 - beta^2) R_hat / (4 pi eps0 |R|^2 (1 - beta^2 sin^2 psi)^(3/2)),
    psi the angle between R and the velocity; B = beta x E / c.
    """
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    r = np.linalg.norm(R)
    sin2 = (R[0] ** 2 + R[1] ** 2) / r ** 2
    # 1 - beta^2 = 1/gamma^2 and 1 - beta^2 sin^2 = cos^2 + sin^2/gamma^2, written
    # this way so that the reference keeps its digits at large gamma
    one_minus_b2 = 1.0 / gamma ** 2
    E = KE * q * one_minus_b2 * (R / r) / (r ** 2 * ((1.0 - sin2) + sin2 * one_minus_b2) ** 1.5)
    B = np.cross(np.array([0.0, 0.0, beta]), E) / C0
    return E, B


@pytest.mark.parametrize("gamma", [1.0 + 1e-9, 2.0, 10.0, 200.0])
@pytest.mark.parametrize("direction", [(0, 0, 1), (1, 0, 0), (0.3, -0.4, 0.5), (0, 1, -2)])
def test_single_pair_matches_moving_charge(gamma, direction):
    q = -1.6e-19
    d = np.asarray(direction, dtype=np.float64)
    d = 1.7e-4 * d / np.linalg.norm(d)
    x = np.array([[0.0, 0.0, 0.0], d])
    p = np.zeros((2, 3))
    p[:, 2] = math.sqrt(gamma ** 2 - 1.0)
    E, B = physics.direct_fields(x, p, np.full(2, q))
    E0, B0 = _moving_charge_field(q, gamma, x[0] - x[1])
    np.testing.assert_allclose(E[0].numpy(), E0, rtol=1e-12, atol=1e-12 * np.abs(E0).max())
    np.testing.assert_allclose(B[0].numpy(), B0, rtol=1e-12, atol=1e-12 * np.abs(E0).max() / C0)
    # g is odd: the partner sees the opposite field
    np.testing.assert_allclose(E[1].numpy(), -E0, rtol=1e-12, atol=1e-12 * np.abs(E0).max())


def test_coulomb_cube_corner():
    """p = 0 (gamma = 1): eight charges on a cube, field at a corner in closed form."""
    a, q = 2.0e-4, 1.0e-15
    corners = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=np.float64) * a
    E, B = physics.direct_fields(corners, np.zeros((8, 3)), np.full(8, q))
    c = 1.0 + 1.0 / math.sqrt(2.0) + 1.0 / (3.0 * math.sqrt(3.0))
    expect = -KE * q / a ** 2 * c * np.ones(3)
    np.testing.assert_allclose(E[0].numpy(), expect, rtol=1e-13)
    assert float(B.abs().max()) == 0.0


def test_monoenergetic_beam_is_boosted_coulomb():
    """Equal momenta along z: lab field = Lorentz-transformed rest-frame Coulomb field."""
    N, gamma, q = 300, 37.0, -1.6e-19
    rng = np.random.default_rng(5)
    x = rng.standard_normal((N, 3)) * np.array([1e-4, 2e-4, 3e-5])
    p = np.zeros((N, 3))
    p[:, 2] = math.sqrt(gamma ** 2 - 1.0)
    E, B = physics.direct_fields(x, p, np.full(N, q))
    # rest frame: z stretched by gamma, plain Coulomb sum
    xr = x * np.array([1.0, 1.0, gamma])
    R = xr[:, None, :] - xr[None, :, :]
    r = np.sqrt((R ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    Er = KE * q * (R / r[..., None] ** 3).sum(1)
    El = Er * np.array([gamma, gamma, 1.0])          # E_perp = gamma E'_perp, E_par = E'_par
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    Bl = np.cross(np.array([0.0, 0.0, beta]), El) / C0
    np.testing.assert_allclose(E.numpy(), El, rtol=1e-10, atol=1e-12 * np.abs(El).max())
    np.testing.assert_allclose(B.numpy(), Bl, rtol=1e-10, atol=1e-12 * np.abs(Bl).max())
    # the exact uniform-motion field agrees when all momenta are equal
    Eu, Bu = physics.uniform_motion_fields(x, p, np.full(N, q))
    np.testing.assert_allclose(Eu.numpy(), El, rtol=1e-10, atol=1e-12 * np.abs(El).max())


def test_uniform_motion_differs_with_spread():
    """With energy spread the paper's kernel is an approximation of the exact field."""
    x, p, q = random_beam(200, seed=3, gamma=10.0, spread=0.1)
    E, _ = physics.direct_fields(x, p, q)
    Eu, _ = physics.uniform_motion_fields(x, p, q)
    rel = float(((E - Eu) ** 2).sum().sqrt() / (Eu ** 2).sum().sqrt())
    assert 1e-6 < rel < 0.5


def test_momentum_conservation():
    """sum_i a_i E_i = 0: g is odd and a_i a_j symmetric (any charges, any momenta)."""
    x, p, q = random_beam(400, seed=11, gamma=5.0, spread=0.2, angle=0.1)
    q = q * (1.0 + np.random.default_rng(1).random(400))
    E, _ = physics.direct_fields(x, p, q)
    a = q * physics.lorentz_gamma(p).numpy()
    tot = (a[:, None] * E.numpy()).sum(0)
    scale = (np.abs(a)[:, None] * np.abs(E.numpy())).sum(0)
    assert np.all(np.abs(tot) <= 1e-12 * scale)


def test_permutation_and_translation_invariance():
    x, p, q = random_beam(256, seed=2)
    E, B = physics.direct_fields(x, p, q)
    perm = np.random.default_rng(0).permutation(256)
    Ep, Bp = physics.direct_fields(x[perm], p[perm], q[perm])
    np.testing.assert_allclose(Ep.numpy(), E.numpy()[perm], rtol=1e-12, atol=1e-14 * float(E.abs().max()))
    shift = np.array([1e-3, -2e-3, 5e-4])
    Et, Bt = physics.direct_fields(x + shift, p, q)
    np.testing.assert_allclose(Et.numpy(), E.numpy(), rtol=1e-8, atol=1e-9 * float(E.abs().max()))


def test_fmm_permutation_invariance():
    """The tree depends on positions, not on input order (no ties here)."""
    x, p, q = random_beam(512, seed=4)
    E, B = bldtt.fmm_fields(x, p, q, 3, 32, 0.5)
    perm = np.random.default_rng(9).permutation(512)
    Ep, Bp = bldtt.fmm_fields(x[perm], p[perm], q[perm], 3, 32, 0.5)
    np.testing.assert_allclose(Ep.numpy(), E.numpy()[perm], rtol=1e-11, atol=1e-13 * float(E.abs().max()))


def test_pairwise_sum_and_gamma_bar():
    rng = np.random.default_rng(3)
    v = rng.standard_normal(1000) * 1e3
    assert abs(physics.pairwise_sum(v) - math.fsum(v)) <= 8 * np.spacing(abs(math.fsum(np.abs(v))))
    ints = rng.integers(-1000, 1000, size=777).astype(np.float64)
    assert physics.pairwise_sum(ints) == float(ints.sum())  # exact for small integers
    assert physics.pairwise_sum(np.array([])) == 0.0
    p = np.zeros((10, 3))
    p[:, 2] = math.sqrt(50.0 ** 2 - 1.0)
    assert abs(physics.gamma_bar(p) - 50.0) < 1e-12
    assert physics.gamma_bar(np.zeros((3, 3))) == 1.0
