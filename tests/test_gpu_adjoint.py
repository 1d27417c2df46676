"""Hand-written adjoint against the oracle's gradients, through the C ABI (GPU).

The reference for the adjoint is the exact gradient of the oracle's FMM with
the plan (tree, boxes, lists, gbar) held fixed, by automatic differentiation
(oracle.gradient.fmm_gradient, itself pinned to central finite differences
on the CPU).  FP64 must agree to 1e-10 relative L2 per gradient; FP32 to the
level FP32 rounding of the same operator allows, and within the FMM's
truncation error plus 1e-6 of the direct-sum gradient.
"""
import numpy as np
import pytest
import torch

from oracle import bldtt, gradient
from paper_2302_07567_gb300 import fmm
from paper_2302_07567_gb300.workloads import make_beam, make_weights, random_beam

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(*arrs, dtype=None):
    return [torch.as_tensor(np.ascontiguousarray(a), device=DEV, dtype=dtype) for a in arrs]


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def lattice512():
    """8 x 8 x 8 lattice: equal cluster radii make the traversal's P2P list
    one-directional for some leaf pairs (32 of 448 here), which exercises
    the FP32 fused near field's single-role partners."""
    g = np.arange(8)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float64) * 1e-3
    _, p, q = random_beam(x.shape[0], seed=6, gamma=4.0, spread=0.05, angle=0.05)
    return x, p, q


CASES = {
    "lattice512": lambda: (lattice512(), 3, 8, 0.5),
    "gauss2k": lambda: (make_beam("gauss4k", N=2048), 4, 64, 0.5),
    "ragged1501": lambda: (random_beam(1501, seed=3, gamma=15.0, spread=0.05, angle=0.02), 3, 37, 0.5),
    "cylinder4k": lambda: (make_beam("cylinder64k", N=4096), 6, 128, 0.5),
    "corehalo8k": lambda: (make_beam("corehalo16m", N=8192), 8, 256, 0.5),
    "gauss3k_n5": lambda: (make_beam("gauss4k", N=3000), 5, 64, 0.5),  # a degree without specialised kernels
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    (x, p, q), n, leaf, eta = CASES[request.param]()
    N = x.shape[0]
    wE, wB = make_weights(N)
    plan = bldtt.build_plan(x, p, n, leaf, eta)
    L, gx, gp, gq = gradient.fmm_gradient(x, p, q, wE, wB, plan)
    return dict(x=x, p=p, q=q, n=n, leaf=leaf, eta=eta, wE=wE, wB=wB, ref=(gx.numpy(), gp.numpy(), gq.numpy()),
                plan=plan)


def gpu_grad(c, prec, flags=0):
    N = c["x"].shape[0]
    odt = torch.float32 if prec == "fp32" else torch.float64
    X, Pm, Q = dev(c["x"], c["p"], c["q"])
    WE, WB = dev(c["wE"], c["wB"], dtype=odt)
    plan = fmm.Plan(N, c["n"], c["leaf"], c["eta"], precision=prec, flags=flags)
    plan.field(X, Pm, Q)
    dx, dp, dq = plan.adjoint(X, Pm, Q, WE, WB)
    torch.cuda.synchronize()
    return plan, dx.cpu().numpy(), dp.cpu().numpy(), dq.cpu().numpy()


def test_lattice_case_has_one_directional_p2p_pairs():
    (x, p, q), n, leaf, eta = CASES["lattice512"]()
    pairs = set(map(tuple, bldtt.build_plan(x, p, n, leaf, eta).p2p))
    assert sum((b, a) not in pairs for a, b in pairs) > 0


def test_adjoint_fp64_matches_oracle_gradient(case):
    _, dx, dp, dq = gpu_grad(case, "fp64")
    gx, gp, gq = case["ref"]
    assert rel(dx, gx) < 1e-10, rel(dx, gx)
    assert rel(dp, gp) < 1e-10, rel(dp, gp)
    assert rel(dq, gq) < 1e-10, rel(dq, gq)


def test_adjoint_fp32_matches_oracle_gradient(case):
    _, dx, dp, dq = gpu_grad(case, "fp32")
    gx, gp, gq = case["ref"]
    for a, b in ((dx, gx), (dp, gp), (dq, gq)):
        assert rel(a, b) < 2e-5, rel(a, b)


def test_second_adjoint_recomputes_and_matches(case):
    """A second adjoint call on one forward recomputes the overwritten locals."""
    N = case["x"].shape[0]
    X, Pm, Q = dev(case["x"], case["p"], case["q"])
    WE, WB = dev(case["wE"], case["wB"])
    plan = fmm.Plan(N, case["n"], case["leaf"], case["eta"], precision="fp64")
    plan.field(X, Pm, Q)
    a = [t.clone() for t in plan.adjoint(X, Pm, Q, WE, WB)]
    b = plan.adjoint(X, Pm, Q, WE, WB)
    c = [t.clone() for t in plan.adjoint(X, Pm, Q, 2.0 * WE, 2.0 * WB)]
    for u, v, w in zip(a, b, c):
        assert torch.equal(u, v)
        assert float((w - 2.0 * u).norm() / u.norm()) < 1e-13
    # linearity in the weights: adjoint(wE, 0) + adjoint(0, wB) = adjoint(wE, wB)
    e = plan.adjoint(X, Pm, Q, WE, torch.zeros_like(WB))
    e = [t.clone() for t in e]
    f = plan.adjoint(X, Pm, Q, torch.zeros_like(WE), WB)
    for u, v, w in zip(a, e, f):
        assert float((v + w - u).norm() / u.norm()) < 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_recompute_mode_matches_oracle_and_default(case, prec, tol):
    """FMM_RECOMPUTE keeps one set of expansions: W and Lambda overwrite the
    locals and multipoles, the target-side far field reads the locals before
    the far-field chain (FP32: in a kernel of its own, after which the near
    field runs beside the chain; FP64: inside the near-field kernel, which
    runs first), and a second adjoint recomputes the upward pass, M2L and
    L2L.  Its
    gradients equal those of the default plan bit for bit (every sum keeps
    its order) and so match the oracle's frozen-plan gradient."""
    plan, dx, dp, dq = gpu_grad(case, prec, flags=fmm.FMM_RECOMPUTE)
    _, ex, ep, eq = gpu_grad(case, prec)
    gx, gp, gq = case["ref"]
    for a, d, b in ((dx, ex, gx), (dp, ep, gp), (dq, eq, gq)):
        np.testing.assert_array_equal(a, d)
        assert rel(a, b) < tol, rel(a, b)
    N = case["x"].shape[0]
    X, Pm, Q = dev(case["x"], case["p"], case["q"])
    odt = plan.out_dtype
    WE, WB = dev(case["wE"], case["wB"], dtype=odt)
    if plan.stats()["kappa"] > 0:  # the adjoint overwrote the expansions: no export
        with pytest.raises(fmm.FMMError):
            plan.export("local")
    again = plan.adjoint(X, Pm, Q, WE, WB)  # recomputes the locals first
    for a, d in zip(again, (dx, dp, dq)):
        np.testing.assert_array_equal(a.cpu().numpy(), d)
    plan.field(X, Pm, Q)
    assert plan.export("local").shape[0] == plan.stats()["nodes"]


def test_recompute_mode_shrinks_the_workspace():
    N = 1 << 16
    small = fmm.Plan(N, 8, 256, 0.5, precision="fp32", flags=fmm.FMM_RECOMPUTE).workspace_bytes
    full = fmm.Plan(N, 8, 256, 0.5, precision="fp32").workspace_bytes
    C, m = (1 << 9) - 1, 9 ** 3
    assert full - small >= (C + 1) * 10 * m * 4  # W (6 m) and Lambda (4 m) floats per cluster


def test_fp32_adjoint_within_truncation_of_direct_gradient():
    x, p, q = make_beam("gauss256k", N=4096)
    wE, wB = make_weights(4096)
    n, leaf, eta = 6, 128, 0.5
    plan = bldtt.build_plan(x, p, n, leaf, eta)
    _, fx, fp_, fq = gradient.fmm_gradient(x, p, q, wE, wB, plan)
    _, dxr, dpr, dqr = gradient.direct_gradient(x, p, q, wE, wB, gbar=plan.tree.gbar)
    c = dict(x=x, p=p, q=q, n=n, leaf=leaf, eta=eta, wE=wE, wB=wB)
    _, dx, dp, dq = gpu_grad(c, "fp32")
    for gpu, fmm_ref, direct in ((dx, fx, dxr), (dp, fp_, dpr), (dq, fq, dqr)):
        trunc = rel(fmm_ref.numpy(), direct.numpy())
        assert rel(gpu, direct.numpy()) <= trunc + 1e-6, (rel(gpu, direct.numpy()), trunc)


def test_autograd_function_backward_is_the_adjoint():
    x, p, q = make_beam("gauss4k", N=3000)
    wE, wB = make_weights(3000)
    X, Pm, Q = dev(x, p, q)
    WE, WB = dev(wE, wB, dtype=torch.float32)
    plan = fmm.Plan(3000, 4, 64, 0.5, precision="fp32")
    Xr, Pr, Qr = (t.clone().requires_grad_(True) for t in (X, Pm, Q))
    E, B = fmm.FMMField.apply(Xr, Pr, Qr, plan)
    loss = (E * WE).sum() + (B * WB).sum()
    loss.backward()
    plan.field(X, Pm, Q)
    dx, dp, dq = plan.adjoint(X, Pm, Q, WE, WB)
    assert torch.allclose(Xr.grad, dx, rtol=0, atol=0)
    assert torch.allclose(Pr.grad, dp, rtol=0, atol=0)
    assert torch.allclose(Qr.grad, dq, rtol=0, atol=0)


GBAR_CASES = {
    "gauss2k": CASES["gauss2k"],
    "ragged1501": CASES["ragged1501"],
    "cylinder4k": CASES["cylinder4k"],
    "single40": lambda: (random_beam(40, seed=4, gamma=5.0, spread=0.1, angle=0.2), 3, 64, 0.5),  # one leaf
}


@pytest.mark.parametrize("name", list(GBAR_CASES))
def test_gbar_term_matches_oracle(name):
    """FMM_GBAR_TERM: gbar follows p (Section 3, gbar = sqrt(1 + pbar.pbar)).
    The full gradient against the oracle's with the same plan and gbar live;
    the gbar term alone (live minus fixed) against the oracle's difference."""
    (x, p, q), n, leaf, eta = GBAR_CASES[name]()
    N = x.shape[0]
    wE, wB = make_weights(N)
    plan = bldtt.build_plan(x, p, n, leaf, eta)
    _, gx, gp, gq = gradient.fmm_gradient(x, p, q, wE, wB, plan, gbar_term=True)
    _, fx, fp, fq = gradient.fmm_gradient(x, p, q, wE, wB, plan)
    want = (gp - fp).numpy()
    assert np.linalg.norm(want) > 1e-8 * np.linalg.norm(gp.numpy())
    c = dict(x=x, p=p, q=q, n=n, leaf=leaf, eta=eta, wE=wE, wB=wB)
    for prec, tol, ttol in (("fp64", 1e-10, 1e-8), ("fp32", 2e-5, 1e-3)):
        _, dx, dp, dq = gpu_grad(c, prec, flags=fmm.FMM_GBAR_TERM)
        assert rel(dx, gx.numpy()) < tol, (prec, rel(dx, gx.numpy()))
        assert rel(dp, gp.numpy()) < tol, (prec, rel(dp, gp.numpy()))
        assert rel(dq, gq.numpy()) < tol, (prec, rel(dq, gq.numpy()))
        _, dx0, dp0, dq0 = gpu_grad(c, prec)
        assert rel(dp - dp0, want) < ttol, (prec, rel(dp - dp0, want))
        # one set of expansions (FMM_RECOMPUTE): Lambda keeps its own buffer
        # beside the multipoles the gbar term reads; the same gradients
        _, rx, rp, rq = gpu_grad(c, prec, flags=fmm.FMM_GBAR_TERM | fmm.FMM_RECOMPUTE)
        for a, b in ((rx, dx), (rp, dp), (rq, dq)):
            np.testing.assert_array_equal(a, b)
