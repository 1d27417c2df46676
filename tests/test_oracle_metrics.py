"""Pins of the error measure of Eq. 5.1 (oracle/metrics.py).

Every parity threshold of the GPU tests goes through field_error, so the
measure itself is pinned here to hand-computed values.  The cases are chosen
so that the plausible slips each fail one of them:
- a dropped square root (0.5 would read 0.25),
- a mean, a sum or a min over {E, B} instead of the max,
- normalising per row or per component instead of over the whole field,
- swapping the test and reference arguments (the denominator is the
  reference's norm).
"""
import numpy as np
import pytest

from oracle import metrics

# E: reference rows (3, 0, 0) and (0, 4, 0), |E_b|^2 = 25.  The test field
# differs by 2.5 in the first row only: |dE|^2 = 6.25, so the relative L2
# error is sqrt(6.25 / 25) = 1/2 exactly.  Per row the errors would be 5/6
# and 0 (mean 5/12, max 5/6); per component (x: 2.5/3, y: 0) likewise.
E_REF = np.array([[3.0, 0.0, 0.0], [0.0, 4.0, 0.0]])
E_TEST = np.array([[5.5, 0.0, 0.0], [0.0, 4.0, 0.0]])
# B: reference rows (1, 2, 2) and (0, 0, 0), |B_b|^2 = 9.  The test field
# differs by 0.75 in the z component of the first row: sqrt(0.5625 / 9) = 1/4.
B_REF = np.array([[1.0, 2.0, 2.0], [0.0, 0.0, 0.0]])
B_TEST = np.array([[1.0, 2.0, 2.75], [0.0, 0.0, 0.0]])


def test_rel_l2_hand_values():
    assert metrics.rel_l2(E_TEST, E_REF) == 0.5
    assert metrics.rel_l2(B_TEST, B_REF) == 0.25
    # the denominator is the reference's norm: swapping the arguments gives
    # sqrt(6.25 / (5.5^2 + 4^2)) = 2.5 / sqrt(46.25), not 1/2
    assert metrics.rel_l2(E_REF, E_TEST) == pytest.approx(2.5 / np.sqrt(46.25), rel=1e-15)


def test_field_error_is_the_max_over_E_and_B():
    assert metrics.field_error(E_TEST, B_TEST, E_REF, B_REF) == 0.5
    # with the roles of the two fields exchanged the max is still 1/2
    assert metrics.field_error(B_TEST, E_TEST, B_REF, E_REF) == 0.5
    # an exact B leaves the E error, an exact E the B error
    assert metrics.field_error(E_TEST, B_REF, E_REF, B_REF) == 0.5
    assert metrics.field_error(E_REF, B_TEST, E_REF, B_REF) == 0.25


def test_zero_reference():
    z = np.zeros((4, 3))
    assert metrics.rel_l2(z, z) == 0.0
    assert metrics.rel_l2(z + 1.0, z) == float("inf")


def test_random_case_against_the_written_formula():
    rng = np.random.default_rng(507567)
    Eb, Bb = rng.standard_normal((2, 1000, 3))
    Et = Eb + 1e-3 * rng.standard_normal((1000, 3))
    Bt = Bb + 3e-3 * rng.standard_normal((1000, 3))
    # Eq. 5.1 written out: sqrt(sum_i |f_i^t - f_i^b|^2 / sum_i |f_i^b|^2)
    eE = np.sqrt(sum(np.dot(Et[i] - Eb[i], Et[i] - Eb[i]) for i in range(1000)) /
                 sum(np.dot(Eb[i], Eb[i]) for i in range(1000)))
    eB = np.sqrt(sum(np.dot(Bt[i] - Bb[i], Bt[i] - Bb[i]) for i in range(1000)) /
                 sum(np.dot(Bb[i], Bb[i]) for i in range(1000)))
    assert metrics.rel_l2(Et, Eb) == pytest.approx(eE, rel=1e-12)
    assert metrics.field_error(Et, Bt, Eb, Bb) == pytest.approx(max(eE, eB), rel=1e-12)
    # the relative error does not change when both fields are scaled by one factor
    assert metrics.rel_l2(1e7 * Et, 1e7 * Eb) == pytest.approx(eE, rel=1e-12)
