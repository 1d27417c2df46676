"""CUDA path against the FP64 CPU oracle, through the C ABI (GPU).

Discrete results (gbar, tree membership, boxes, split axes, interaction
lists) must match the oracle bit for bit.  Floating-point results: the FP64
build within 1e-12 relative L2 (Eq. 5.1) of the oracle's FMM; the FP32 build
within 1e-5 of the oracle's FMM (FP32 rounding of the same algorithm) and
within the FMM's own truncation error plus 1e-6 of the brute force.
"""
import numpy as np
import pytest
import torch

from oracle import bldtt, gradient, metrics, physics
from paper_2302_07567_gb300 import fmm
from paper_2302_07567_gb300.workloads import make_beam, make_weights, random_beam

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(*arrs):
    return [torch.as_tensor(np.ascontiguousarray(a), device=DEV) for a in arrs]


def run(x, p, q, n, leaf, eta, prec, flags=0):
    plan = fmm.Plan(len(x), n, leaf, eta, precision=prec, flags=flags)
    E, B = plan.field(*dev(x, p, q))
    torch.cuda.synchronize()
    return plan, E.double().cpu().numpy(), B.double().cpu().numpy()


def _ties(N, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 6, size=(N, 3)).astype(np.float64) * 1e-4
    x += rng.integers(0, 2, size=(N, 1)) * 1e-9  # few distinct values, many exact ties
    p = np.zeros((N, 3))
    p[:, 2] = 3.0
    return x, p, np.full(N, -1.6e-19)


CASES = {
    "gauss4k": lambda: (make_beam("gauss4k"), 4, 64, 0.5),
    "ragged3001": lambda: (random_beam(3001, seed=1, gamma=20.0, spread=0.05, angle=0.01), 3, 37, 0.6),
    "cylinder8k": lambda: (make_beam("cylinder64k", N=8192), 6, 128, 0.5),
    "ties": lambda: (_ties(2000, 3), 2, 16, 0.5),
    "small_leafless": lambda: (random_beam(50, seed=5), 4, 64, 0.5),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    (x, p, q), n, leaf, eta = CASES[request.param]()
    ref_plan = bldtt.build_plan(x, p, n, leaf, eta)
    ref = bldtt.fmm_stages(x, p, q, ref_plan)
    return dict(name=request.param, x=x, p=p, q=q, n=n, leaf=leaf, eta=eta, ref_plan=ref_plan, ref=ref)


@pytest.fixture(scope="module")
def gpu64(case):
    return run(case["x"], case["p"], case["q"], case["n"], case["leaf"], case["eta"], "fp64")


def test_gbar_is_bit_exact(case, gpu64):
    plan = gpu64[0]
    assert plan.export("gbar")[0] == case["ref_plan"].tree.gbar


def test_tree_is_bit_exact(case, gpu64):
    plan = gpu64[0]
    tr = case["ref_plan"].tree
    C = tr.C
    nodes, bbox, axis, perm = plan.export("nodes"), plan.export("bbox"), plan.export("axis"), plan.export("perm")
    assert nodes.shape == (C, 2)
    np.testing.assert_array_equal(bbox[:, :3], tr.lo[1:])
    np.testing.assert_array_equal(bbox[:, 3:], tr.hi[1:])
    np.testing.assert_array_equal(axis, tr.axis[1:])
    for i in range(1, C + 1):
        st, cnt = nodes[i - 1]
        assert cnt == tr.members[i].size
        if tr.is_leaf(i):
            np.testing.assert_array_equal(np.sort(perm[st:st + cnt]), np.sort(tr.members[i]))


def test_interaction_lists_are_exact(case, gpu64):
    plan = gpu64[0]
    rp = case["ref_plan"]
    p2p = plan.export("p2p")
    m2l = plan.export("m2l")
    np.testing.assert_array_equal(p2p, np.array(sorted(rp.p2p), dtype=np.int32).reshape(-1, 2))
    np.testing.assert_array_equal(m2l, np.array(sorted(rp.m2l), dtype=np.int32).reshape(-1, 2))
    st = plan.stats()
    assert st["p2p_pairs"] == len(rp.p2p) and st["m2l_pairs"] == len(rp.m2l)
    sizes = plan.export("nodes")[:, 1].astype(np.float64)
    cover = sum(sizes[t - 1] * sizes[s - 1] for t, s in np.concatenate([p2p, m2l]))
    assert cover == float(len(case["x"])) ** 2


def _node_rel(a, b):
    num = np.sqrt(((a - b) ** 2).sum(axis=(1, 2)))
    den = np.sqrt((b ** 2).sum(axis=(1, 2)))
    return np.where(den > 0, num / np.where(den > 0, den, 1), num)


def test_p2p_interactions_counted_on_device(case, gpu64):
    """stats()["p2p_interactions"] (sum |S_t||S_s| over the P2P list minus the
    N self pairs, summed by the traversal kernel) against the exported list."""
    plan = gpu64[0]
    cnt = plan.export("nodes")[:, 1].astype(np.int64)
    pairs = plan.export("p2p").astype(np.int64)
    total = int(np.sum(cnt[pairs[:, 0] - 1] * cnt[pairs[:, 1] - 1])) - len(case["x"])
    assert plan.stats()["p2p_interactions"] == total


def test_multipoles_and_locals_fp64(case, gpu64):
    plan = gpu64[0]
    ref, rp = case["ref"], case["ref_plan"]
    C = rp.tree.C
    Mref = np.stack([ref["M"][i].numpy().T for i in range(1, C + 1)])
    Mg = plan.export("multipole")
    assert _node_rel(Mg, Mref).max() < 1e-12
    if rp.tree.kappa > 0:
        Lref = np.stack([ref["L"][i].numpy().T for i in range(1, C + 1)])
        Lg = plan.export("local")
        scale = np.sqrt((Lref ** 2).sum(axis=(1, 2))).max()
        err = np.sqrt(((Lg - Lref) ** 2).sum(axis=(1, 2)))
        assert err.max() < 1e-12 * scale


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8])
def test_multipoles_fp32(n):
    """FP32 multipoles (Alg. 3 at the leaves, the separable kernel for 3, 5,
    7 and 9 points per axis, the point-per-thread one for 4; Alg. 5 above)
    node by node within FP32 rounding of the oracle's."""
    x, p, q = make_beam("gauss4k", N=3000)
    leaf = 64
    rp = bldtt.build_plan(x, p, n, leaf, 0.5)
    ref = bldtt.fmm_stages(x, p, q, rp)
    plan, _, _ = run(x, p, q, n, leaf, 0.5, "fp32")
    C = rp.tree.C
    Mref = np.stack([ref["M"][i].numpy().T for i in range(1, C + 1)])
    Mg = plan.export("multipole").astype(np.float64)
    assert Mg.shape == Mref.shape
    assert _node_rel(Mg, Mref).max() < 2e-6


def test_fields_fp64_match_oracle_fmm(case, gpu64):
    _, E, B = gpu64
    ref = case["ref"]
    assert metrics.field_error(E, B, ref["E"].numpy(), ref["B"].numpy()) < 1e-12


def test_fields_fp32(case):
    x, p, q = case["x"], case["p"], case["q"]
    _, E, B = run(x, p, q, case["n"], case["leaf"], case["eta"], "fp32")
    ref = case["ref"]
    e_alg = metrics.field_error(E, B, ref["E"].numpy(), ref["B"].numpy())
    assert e_alg < 1e-5, e_alg
    Ed, Bd = physics.direct_fields(x, p, q)
    e_trunc = metrics.field_error(ref["E"].numpy(), ref["B"].numpy(), Ed.numpy(), Bd.numpy())
    e32 = metrics.field_error(E, B, Ed.numpy(), Bd.numpy())
    assert e32 <= e_trunc + 1e-6, (e32, e_trunc)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_eta_to_zero_is_brute_force(prec, tol):
    x, p, q = random_beam(3000, seed=21, gamma=5.0)
    plan, E, B = run(x, p, q, 4, 40, 1e-30, prec)
    assert plan.stats()["m2l_pairs"] == 0
    Ed, Bd = physics.direct_fields(x, p, q)
    assert metrics.field_error(E, B, Ed.numpy(), Bd.numpy()) < tol


def test_direct_field_matches_oracle():
    x, p, q = make_beam("gauss4k")
    gb = physics.gamma_bar(p)
    tg = np.arange(0, 4096, 7)
    E, B = fmm.direct_field(*dev(x, p, q), gbar=gb, targets=torch.as_tensor(tg, device=DEV))
    Ed, Bd = physics.direct_fields(x, p, q, targets=tg, gbar=gb)
    assert metrics.field_error(E.cpu().numpy(), B.cpu().numpy(), Ed.numpy(), Bd.numpy()) < 1e-13


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_runs_are_bitwise_deterministic(prec):
    x, p, q = make_beam("cylinder64k", N=20000)
    plan = fmm.Plan(20000, 6, 128, 0.5, precision=prec)
    X, Pm, Q = dev(x, p, q)
    E1, B1 = plan.field(X, Pm, Q)
    E1, B1 = E1.clone(), B1.clone()
    E2, B2 = plan.field(X, Pm, Q)
    assert torch.equal(E1, E2) and torch.equal(B1, B2)


@pytest.mark.parametrize("prec,n,leaf", [("fp32", 8, 256), ("fp32", 6, 128), ("fp64", 4, 64)])
def test_serial_stage_order_is_bitwise_equal(prec, n, leaf):
    """FMM_SERIAL runs the independent branches one after another on one
    stream; every sum keeps its order, so fields and gradients are equal."""
    N = 20000
    x, p, q = make_beam("corehalo16m", N=N)
    wE, wB = make_weights(N)
    X, Pm, Q = dev(x, p, q)
    out = []
    for flags in (0, fmm.FMM_SERIAL):
        plan = fmm.Plan(N, n, leaf, 0.5, precision=prec, flags=flags)
        E, B = plan.field(X, Pm, Q)
        WE, WB = (torch.as_tensor(w, device=DEV, dtype=plan.out_dtype) for w in (wE, wB))
        out.append([E, B, *plan.adjoint(X, Pm, Q, WE, WB)])
        plan.close()
    for a, b in zip(*out):
        assert torch.equal(a, b)


def test_edge_cases():
    # one particle: no field
    x, p, q = random_beam(1, seed=0)
    _, E, B = run(x, p, q, 3, 8, 0.5, "fp64")
    assert np.all(E == 0) and np.all(B == 0)
    # two particles: the moving-charge closed form through the library
    x = np.array([[0.0, 0.0, 0.0], [1e-4, 2e-4, -3e-5]])
    p = np.zeros((2, 3))
    p[:, 2] = np.sqrt(30.0 ** 2 - 1.0)
    q = np.full(2, -1.6e-19)
    _, E, B = run(x, p, q, 3, 8, 0.5, "fp64")
    Ed, Bd = physics.direct_fields(x, p, q)
    np.testing.assert_allclose(E, Ed.numpy(), rtol=1e-13)
    # all particles in one z plane (zero-width boxes), with coincident pairs
    rng = np.random.default_rng(4)
    x = rng.standard_normal((600, 3)) * 1e-3
    x[:, 2] = 2e-4
    x[300:310] = x[290:300]
    p = np.zeros((600, 3))
    p[:, 2] = 5.0
    q = np.full(600, -1.6e-19)
    for n in (3, 4):  # 4: the separable P2M and the paired M2L kernels on zero-width boxes
        Er, Br = bldtt.fmm_fields(x, p, q, n, 16, 0.5)
        for prec, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
            _, E, B = run(x, p, q, n, 16, 0.5, prec)
            assert np.all(np.isfinite(E)) and np.all(np.isfinite(B))
            assert metrics.field_error(E, B, Er.numpy(), Br.numpy()) < tol
    # and the FP32 adjoint there (the far-field basis derivatives of a zero-width side)
    wE, wB = make_weights(600)
    ref_plan = bldtt.build_plan(x, p, 4, 16, 0.5)
    _, gx, gp, gq = gradient.fmm_gradient(x, p, q, wE, wB, ref_plan)
    plan = fmm.Plan(600, 4, 16, 0.5, precision="fp32")
    X, P, Q = dev(x, p, q)
    plan.field(X, P, Q)
    WE, WB = (torch.as_tensor(a, device=DEV, dtype=torch.float32) for a in (wE, wB))
    for a, b in zip(plan.adjoint(X, P, Q, WE, WB), (gx, gp, gq)):
        a, b = a.cpu().numpy(), b.numpy()
        assert np.all(np.isfinite(a)) and np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-5


def test_nonfinite_input_is_rejected():
    x, p, q = random_beam(500, seed=2)
    x[17, 1] = np.nan
    plan = fmm.Plan(500, 3, 16, 0.5, precision="fp32")
    with pytest.raises(fmm.FMMError) as ei:
        plan.field(*dev(x, p, q))
    assert ei.value.status == fmm.FMM_ENONFINITE


def test_list_overflow_grows_and_matches():
    x, p, q = make_beam("gauss4k")
    plan = fmm.Plan(4096, 4, 64, 0.5, precision="fp64", capacity=(8, 8, 16))
    E, B = plan.field(*dev(x, p, q))
    st = plan.stats()
    assert st["cap_p2p"] >= st["p2p_pairs"] > 8
    _, E2, B2 = run(x, p, q, 4, 64, 0.5, "fp64")
    np.testing.assert_array_equal(E.cpu().numpy(), E2)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bounds_check_mode_passes_and_changes_nothing(case, prec):
    """FMM_BOUNDS_CHECK verifies the tables, the leaf order and both lists
    (including sum |S_t||S_s| = N^2) and must not change any result."""
    x, p, q = case["x"], case["p"], case["q"]
    N = len(x)
    X, Pm, Q = dev(x, p, q)
    odt = torch.float32 if prec == "fp32" else torch.float64
    rng = np.random.default_rng(11)
    WE, WB = (torch.as_tensor(rng.standard_normal((N, 3)), device=DEV, dtype=odt) for _ in range(2))
    out = []
    for flags in (0, fmm.FMM_BOUNDS_CHECK):
        plan = fmm.Plan(N, case["n"], case["leaf"], case["eta"], precision=prec, flags=flags)
        E, B = plan.field(X, Pm, Q)
        E, B = E.clone(), B.clone()
        grads = [t.clone() for t in plan.adjoint(X, Pm, Q, WE, WB)]
        out.append((E, B, *grads))
    for a, b in zip(*out):
        assert torch.equal(a, b)


SIZE_AWARE_CASES = {
    "gauss4k_n4": lambda: (make_beam("gauss4k"), 4, 64, 0.5),
    "ragged3001_n3": lambda: (random_beam(3001, seed=1, gamma=20.0, spread=0.05, angle=0.01), 3, 37, 0.5),
    "cylinder8k_n3": lambda: (make_beam("cylinder64k", N=8192), 3, 32, 0.5),
}


@pytest.mark.parametrize("name", list(SIZE_AWARE_CASES))
def test_size_aware_variant_matches_oracle(name):
    """FMM_SIZE_AWARE: admissible pairs below m^2 particle pairs go to P2P.  The
    lists equal the oracle's size-aware plan, FP64 fields and gradients match
    its FMM, and the error against the brute force does not grow."""
    (x, p, q), n, leaf, eta = SIZE_AWARE_CASES[name]()
    N = len(x)
    ref = bldtt.build_plan(x, p, n, leaf, eta, size_aware=True)
    plain = bldtt.build_plan(x, p, n, leaf, eta)
    assert len(ref.m2l) < len(plain.m2l)
    X, Pm, Q = dev(x, p, q)
    plan = fmm.Plan(N, n, leaf, eta, precision="fp64", flags=fmm.FMM_SIZE_AWARE)
    E, B = plan.field(X, Pm, Q)
    np.testing.assert_array_equal(plan.export("p2p"), np.array(sorted(ref.p2p), dtype=np.int32))
    np.testing.assert_array_equal(plan.export("m2l"), np.array(sorted(ref.m2l), dtype=np.int32).reshape(-1, 2))
    cnt = plan.export("nodes")[:, 1].astype(np.int64)
    pairs = plan.export("p2p").astype(np.int64)
    assert plan.stats()["p2p_interactions"] == int(np.sum(cnt[pairs[:, 0] - 1] * cnt[pairs[:, 1] - 1])) - N
    Er, Br = bldtt.fmm_fields(x, p, q, n, leaf, eta, plan=ref)
    assert metrics.field_error(E.cpu().numpy(), B.cpu().numpy(), Er.numpy(), Br.numpy()) < 1e-12
    rng = np.random.default_rng(5)
    wE, wB = rng.standard_normal((N, 3)), rng.standard_normal((N, 3))
    from oracle import gradient
    _, gx, gp, gq = gradient.fmm_gradient(x, p, q, wE, wB, ref)
    dx, dp, dq = plan.adjoint(X, Pm, Q, *dev(wE, wB))
    for a, b in ((dx, gx), (dp, gp), (dq, gq)):
        a, b = a.cpu().numpy(), b.numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10
    E32, B32 = fmm.Plan(N, n, leaf, eta, precision="fp32", flags=fmm.FMM_SIZE_AWARE).field(X, Pm, Q)
    assert metrics.field_error(E32.double().cpu().numpy(), B32.double().cpu().numpy(), Er.numpy(), Br.numpy()) < 1e-5
    Ed, Bd = physics.direct_fields(x, p, q)
    Ep, Bp = bldtt.fmm_fields(x, p, q, n, leaf, eta, plan=plain)
    e_sa = metrics.field_error(E.cpu().numpy(), B.cpu().numpy(), Ed.numpy(), Bd.numpy())
    e_plain = metrics.field_error(Ep.numpy(), Bp.numpy(), Ed.numpy(), Bd.numpy())
    assert e_sa <= e_plain, (e_sa, e_plain)


@pytest.mark.parametrize("n", [3, 5])
def test_polynomial_test_kernel_is_exact(n):
    """FMM_TEST_POLY_KERNEL: g(R) = R (1 + R_x^2 + R_y^2 + gbar^2 R_z^2) has degree 3
    in each variable, so for n >= 3 every interpolation step is exact (Theorem 1,
    the lemma of Appendix A) and the FMM equals the direct sum of this g to
    rounding, for any eta."""
    x, p, q = random_beam(600, seed=7, gamma=4.0)
    x = x * 1e3  # O(1) coordinates: both terms of 1 + D matter
    plan = fmm.Plan(600, n, 16, 0.9, precision="fp64", flags=fmm.FMM_TEST_POLY_KERNEL)
    E, B = plan.field(*dev(x, p, q))
    st = plan.stats()
    assert st["m2l_pairs"] > 20
    gb = st["gbar"]
    R = x[:, None, :] - x[None, :, :]
    D = R[..., 0] ** 2 + R[..., 1] ** 2 + gb * gb * R[..., 2] ** 2
    g = R * (1.0 + D)[..., None]
    a = q * np.sqrt(1.0 + (p * p).sum(1))
    b = q[:, None] * p
    Ed = physics.KE * np.einsum("j,ijk->ik", a, g)
    Bd = physics.KE / physics.C0 * np.cross(np.broadcast_to(b[None, :, :], g.shape), g).sum(1)
    assert metrics.field_error(E.cpu().numpy(), B.cpu().numpy(), Ed, Bd) < 1e-10
    with pytest.raises(fmm.FMMError):
        fmm.Plan(600, n, 16, 0.9, precision="fp32", flags=fmm.FMM_TEST_POLY_KERNEL)
    with pytest.raises(fmm.FMMError):
        plan.adjoint(*dev(x, p, q), *dev(np.ones((600, 3)), np.ones((600, 3))))
