"""Pins of the oracle's reference gradients against central finite differences (CPU)."""
import numpy as np
import pytest
import torch

from oracle import bldtt, gradient, physics
from paper_2302_07567_gb300.workloads import make_weights, random_beam


def _fd(fun, arr, idx, h):
    a1 = arr.copy()
    a2 = arr.copy()
    a1[idx] += h
    a2[idx] -= h
    return (fun(a1) - fun(a2)) / (2.0 * h)


@pytest.mark.parametrize("which", ["fmm", "direct"])
def test_gradient_matches_central_differences(which):
    N = 96
    x, p, q = random_beam(N, seed=12, gamma=6.0, spread=0.05, angle=0.05)
    wE, wB = make_weights(N)
    plan = bldtt.build_plan(x, p, 4, 8, 0.6)
    gb = plan.tree.gbar
    assert len(plan.m2l) > 0
    if which == "fmm":
        L0, gx, gp, gq = gradient.fmm_gradient(x, p, q, wE, wB, plan)

        def loss(xx, pp, qq):
            E, B = bldtt.fmm_fields(xx, pp, qq, 4, 8, 0.6, plan=plan)
            return gradient.loss_value(E, B, wE, wB)
    else:
        L0, gx, gp, gq = gradient.direct_gradient(x, p, q, wE, wB, gbar=gb)

        def loss(xx, pp, qq):
            E, B = physics.direct_fields(xx, pp, qq, gbar=gb)
            return gradient.loss_value(E, B, wE, wB)

    rng = np.random.default_rng(0)
    for _ in range(6):
        j, k = int(rng.integers(N)), int(rng.integers(3))
        h = 1e-6 * max(abs(x[j, k]), 1e-4)
        fd = _fd(lambda a: loss(a, p, q), x, (j, k), h)
        assert abs(fd - float(gx[j, k])) <= 2e-5 * abs(fd) + 2e-8 * float(gx.abs().max())
        h = 1e-6 * max(abs(p[j, k]), 1e-2)
        fd = _fd(lambda a: loss(x, a, q), p, (j, k), h)
        assert abs(fd - float(gp[j, k])) <= 2e-5 * abs(fd) + 2e-8 * float(gp.abs().max())
        h = 1e-6 * abs(q[j])
        fd = _fd(lambda a: loss(x, p, a), q, (j,), h)
        assert abs(fd - float(gq[j])) <= 2e-5 * abs(fd) + 2e-8 * float(gq.abs().max())


def test_fmm_gradient_approaches_direct_gradient():
    N = 256
    x, p, q = random_beam(N, seed=13, gamma=8.0)
    wE, wB = make_weights(N)
    errs = []
    for n in (2, 5):
        plan = bldtt.build_plan(x, p, n, 16, 0.5)
        _, gx, gp, gq = gradient.fmm_gradient(x, p, q, wE, wB, plan)
        _, dx, dp, dq = gradient.direct_gradient(x, p, q, wE, wB, gbar=plan.tree.gbar)
        errs.append(max(float((gx - dx).norm() / dx.norm()), float((gq - dq).norm() / dq.norm())))
    assert errs[1] < errs[0] < 0.1


def test_sampled_direct_gradient_matches_full_autograd():
    """The per-particle O(N) gradient equals the full direct-sum gradient rows."""
    N = 150
    x, p, q = random_beam(N, seed=14, gamma=7.0, spread=0.05, angle=0.05)
    wE, wB = make_weights(N)
    gb = physics.gamma_bar(p)
    _, gx, gp, gq = gradient.direct_gradient(x, p, q, wE, wB, gbar=gb)
    idx = [0, 17, 88, 149]
    sx, sp, sq = gradient.direct_gradient_at(x, p, q, wE, wB, idx, gb)
    np.testing.assert_allclose(sx.numpy(), gx.numpy()[idx], rtol=1e-10, atol=1e-12 * float(gx.abs().max()))
    np.testing.assert_allclose(sp.numpy(), gp.numpy()[idx], rtol=1e-10, atol=1e-12 * float(gp.abs().max()))
    np.testing.assert_allclose(sq.numpy(), gq.numpy()[idx], rtol=1e-10, atol=1e-12 * float(gq.abs().max()))


@pytest.mark.parametrize("which", ["fmm", "direct"])
def test_gbar_term_matches_central_differences(which):
    """gbar as the function of p of Section 3 (below Eq. 3.2): dL/dp against
    central differences of the loss whose gbar is recomputed from the
    perturbed momenta (tree, boxes and lists of the FMM plan held fixed)."""
    N = 96 if which == "fmm" else 24
    x, p, q = random_beam(N, seed=21, gamma=4.0, spread=0.1, angle=0.2)
    wE, wB = make_weights(N)
    plan = bldtt.build_plan(x, p, 4, 8, 0.6)
    assert len(plan.m2l) > 0
    if which == "fmm":
        _, gx, gp, gq = gradient.fmm_gradient(x, p, q, wE, wB, plan, gbar_term=True)
        _, fx, fp, fq = gradient.fmm_gradient(x, p, q, wE, wB, plan)

        def loss(pp):
            g = physics.gamma_bar(pp)
            E, B = bldtt.fmm_fields(x, pp, q, 4, 8, 0.6, plan=plan, kernel=lambda R, _f: physics.kernel_g(R, g))
            return gradient.loss_value(E, B, wE, wB)
    else:
        _, gx, gp, gq = gradient.direct_gradient(x, p, q, wE, wB, gbar_term=True)
        _, fx, fp, fq = gradient.direct_gradient(x, p, q, wE, wB)

        def loss(pp):
            E, B = physics.direct_fields(x, pp, q)  # gbar from pp
            return gradient.loss_value(E, B, wE, wB)

    rng = np.random.default_rng(1)
    worst_live, worst_frozen = 0.0, 0.0
    for _ in range(8):
        j, k = int(rng.integers(N)), int(rng.integers(3))
        h = 1e-5 * max(abs(p[j, k]), 1e-2)
        fd = _fd(loss, p, (j, k), h)
        tol = 2e-5 * abs(fd) + 2e-8 * float(gp.abs().max())
        worst_live = max(worst_live, abs(fd - float(gp[j, k])) / tol)
        worst_frozen = max(worst_frozen, abs(fd - float(fp[j, k])) / tol)
    assert worst_live <= 1.0, worst_live
    assert worst_frozen > 10.0, worst_frozen  # the gbar term is not negligible here


def test_gbar_term_adds_one_common_vector_to_dp():
    """dL/dp with gbar live minus dL/dp with gbar fixed is, for every particle,
    dL/dgbar * pbar / (N gbar) (chain rule through gbar = sqrt(1 + pbar.pbar));
    dL/dx and dL/dq do not change.  dL/dgbar is taken here by differentiating
    the FMM with respect to gbar alone."""
    N = 128
    x, p, q = random_beam(N, seed=22, gamma=6.0, spread=0.05, angle=0.1)
    wE, wB = make_weights(N)
    plan = bldtt.build_plan(x, p, 3, 16, 0.5)
    _, gx, gp, gq = gradient.fmm_gradient(x, p, q, wE, wB, plan, gbar_term=True)
    _, fx, fp, fq = gradient.fmm_gradient(x, p, q, wE, wB, plan)
    assert torch.equal(gx, fx) and torch.equal(gq, fq)
    dLdg = gradient.fmm_dloss_dgbar(x, p, q, wE, wB, plan)
    pbar = physics.mean_momentum(p)
    want = dLdg * pbar / (N * plan.tree.gbar)
    diff = (gp - fp).numpy()
    np.testing.assert_allclose(diff, np.broadcast_to(want, diff.shape), rtol=1e-9, atol=1e-12 * abs(want).max())
    assert abs(want).max() > 1e-6 * float(fp.abs().max())
