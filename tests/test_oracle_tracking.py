"""Pins of the tracking oracle (oracle/tracking.py; not in the paper).

The Boris step is pinned to what the scheme fixes exactly: a pure electric
field changes u by 2 a E; a pure magnetic field rotates u about B by the
angle 2 atan(|t|) and keeps |u|; with no field x moves by c dt u / gamma.
The refreshed plan is pinned to the plan it comes from (same input: same
boxes; a rigid translation: translated boxes and equal fields), to the
bounding boxes of Section 2, and to the admissibility test it reruns.
"""
import numpy as np
import pytest

from oracle import bldtt, tracking
from oracle.physics import C0
from paper_2302_07567_gb300.workloads import random_beam

ME = 9.1093837015e-31


def _rng(seed=0):
    return np.random.default_rng(2302 + seed)


def test_pure_electric_field_kick():
    r = _rng()
    N = 50
    x, p, E = r.standard_normal((N, 3)), r.standard_normal((N, 3)), 1e5 * r.standard_normal((N, 3))
    q = np.full(N, -1.6e-19)
    dt = 1e-12
    x1, p1 = tracking.boris_push(x, p, q, E, np.zeros((N, 3)), ME, dt)
    a = (q * dt / (2 * ME * C0))[:, None]
    np.testing.assert_allclose(p1, p + 2 * a * E, rtol=1e-14, atol=1e-15)
    g1 = np.sqrt(1 + np.sum(p1 * p1, axis=1))
    np.testing.assert_allclose(x1, x + C0 * dt * p1 / g1[:, None], rtol=1e-14)


def test_pure_magnetic_field_rotates_by_twice_atan_t():
    r = _rng(1)
    N = 40
    p = r.standard_normal((N, 3)) * 5
    B = r.standard_normal((N, 3)) * 2.0
    q = np.full(N, -1.6e-19)
    dt = 3e-12
    _, p1 = tracking.boris_push(np.zeros((N, 3)), p, q, np.zeros((N, 3)), B, ME, dt)
    # |u| is kept
    np.testing.assert_allclose(np.linalg.norm(p1, axis=1), np.linalg.norm(p, axis=1), rtol=1e-13)
    # the component along B is kept, the perpendicular part turns by 2 atan(|t|)
    b = B / np.linalg.norm(B, axis=1, keepdims=True)
    par0, par1 = np.sum(p * b, axis=1), np.sum(p1 * b, axis=1)
    np.testing.assert_allclose(par1, par0, rtol=1e-12, atol=1e-12)
    perp0 = p - par0[:, None] * b
    perp1 = p1 - par1[:, None] * b
    cosang = np.sum(perp0 * perp1, axis=1) / (np.linalg.norm(perp0, axis=1) * np.linalg.norm(perp1, axis=1))
    gamma = np.sqrt(1 + np.sum(p * p, axis=1))
    tmag = np.abs(q) * dt / (2 * ME * gamma) * np.linalg.norm(B, axis=1)
    np.testing.assert_allclose(np.arccos(np.clip(cosang, -1, 1)), 2 * np.arctan(tmag), rtol=1e-9)
    # an electron (q < 0) turns right-handed about B: (perp0 x perp1) . b > 0
    assert np.all(np.sum(np.cross(perp0, perp1) * b, axis=1) > 0)


def test_no_field_drift():
    r = _rng(2)
    N = 30
    x, p = r.standard_normal((N, 3)), r.standard_normal((N, 3)) * 10
    x1, p1 = tracking.boris_push(x, p, np.full(N, 1.0), np.zeros((N, 3)), np.zeros((N, 3)), 1.0, 2e-9)
    np.testing.assert_array_equal(p1, p)
    beta = p / np.sqrt(1 + np.sum(p * p, axis=1))[:, None]
    np.testing.assert_allclose(x1, x + C0 * 2e-9 * beta, rtol=1e-14, atol=1e-14)


def test_refresh_with_same_input_is_the_plan():
    x, p, q = random_beam(1500, seed=7)
    plan = bldtt.build_plan(x, p, 4, 32, 0.5)
    ref, valid = tracking.refresh_plan(plan, x, p)
    assert valid
    np.testing.assert_array_equal(ref.tree.lo, plan.tree.lo)
    np.testing.assert_array_equal(ref.tree.hi, plan.tree.hi)
    assert ref.tree.gbar == plan.tree.gbar and ref.p2p == plan.p2p and ref.m2l == plan.m2l


def test_refresh_after_rigid_translation():
    x, p, q = random_beam(1500, seed=8)
    plan = bldtt.build_plan(x, p, 4, 32, 0.5)
    shift = np.array([0.25e-3, -0.5e-3, 1.0e-3])
    ref, valid = tracking.refresh_plan(plan, x + shift, p)
    assert valid
    for i in range(1, plan.tree.C + 1):
        lo, hi = ref.tree.lo[i], ref.tree.hi[i]
        mem = plan.tree.members[i]
        np.testing.assert_array_equal(lo, (x + shift)[mem].min(axis=0))
        np.testing.assert_array_equal(hi, (x + shift)[mem].max(axis=0))
    E0, B0 = bldtt.fmm_fields(x, p, q, 4, 32, 0.5, plan=plan)
    E1, B1 = bldtt.fmm_fields(x + shift, p, q, 4, 32, 0.5, plan=ref)
    rel = lambda a, b: float(np.linalg.norm(a.numpy() - b.numpy()) / np.linalg.norm(b.numpy()))  # noqa: E731
    assert rel(E1, E0) < 1e-9 and rel(B1, B0) < 1e-9


def test_refresh_detects_an_inadmissible_pair():
    x, p, q = random_beam(1500, seed=9)
    plan = bldtt.build_plan(x, p, 4, 32, 0.5)
    assert len(plan.m2l) > 0
    # move one leaf's particles onto the centre of one of its M2L partners:
    # the two boxes then overlap and the pair cannot stay admissible
    t, s = next((i, j) for i, j in plan.m2l if plan.tree.is_leaf(i))
    x2 = x.copy()
    mem_t = plan.tree.members[t]
    centre_s = 0.5 * (plan.tree.lo[s] + plan.tree.hi[s])
    x2[mem_t] = centre_s + 1e-3 * (x[mem_t] - x[mem_t].mean(axis=0))
    _, valid = tracking.refresh_plan(plan, x2, p)
    assert not valid
