"""Pins of the oracle's serial FMM (Algs. 3-17, Theorem 1, Lemma of Appendix A).

The FMM is checked against facts fixed outside it: the interaction lists
partition every ordered particle pair exactly once; with eta -> 0 every pair
is direct and the FMM is the brute force; with a kernel that is a polynomial
of degree <= n in each variable every interpolation step is exact (Theorem 1
and the cumulative-local Lemma), so the FMM equals the direct sum for any
eta; moments reproduce the particles' total mass and dipole; and the error
against the brute force falls as n grows and as eta shrinks (Section 5).
"""
import numpy as np
import pytest
import torch

from oracle import bldtt, interp, metrics, physics
from paper_2302_07567_gb300.workloads import random_beam


def _coverage(plan):
    N = plan.tree.N
    cover = np.zeros((N, N), dtype=np.int64)
    for t, s in plan.p2p + plan.m2l:
        ti, sj = plan.tree.members[t], plan.tree.members[s]
        cover[np.ix_(ti, sj)] += 1
    return cover


@pytest.mark.parametrize("N,N0,eta,gamma", [(300, 8, 0.5, 10.0), (513, 16, 0.7, 1.0), (1024, 32, 0.4, 50.0),
                                            (64, 64, 0.5, 3.0), (9, 2, 0.9, 2.0)])
def test_lists_partition_all_pairs(N, N0, eta, gamma):
    x, p, q = random_beam(N, seed=N, gamma=gamma)
    plan = bldtt.build_plan(x, p, 3, N0, eta)
    np.testing.assert_array_equal(_coverage(plan), np.ones((N, N), dtype=np.int64))
    tr = plan.tree
    s = (1.0, 1.0, tr.gbar)
    for t, u in plan.p2p:
        assert tr.is_leaf(t) and tr.is_leaf(u)
    for t, u in plan.m2l:
        assert bldtt.admissible(tr.lo[t], tr.hi[t], tr.lo[u], tr.hi[u], s, eta)
    assert len(set(plan.p2p + plan.m2l)) == len(plan.p2p) + len(plan.m2l)


def test_eta_to_zero_is_brute_force():
    x, p, q = random_beam(700, seed=1)
    E, B = bldtt.fmm_fields(x, p, q, 4, 32, 1e-30)
    Ed, Bd = physics.direct_fields(x, p, q)
    assert metrics.field_error(E.numpy(), B.numpy(), Ed.numpy(), Bd.numpy()) < 1e-13


def _poly_kernel(gbar):
    def g(R, gb):
        D = R[..., 0] ** 2 + R[..., 1] ** 2 + (gb * gb) * R[..., 2] ** 2
        return R * (1.0 + D)[..., None] * 1e6
    return g


@pytest.mark.parametrize("n", [3, 5])
def test_polynomial_kernel_is_exact(n):
    """g_poly(x, y) = (x - y)(1 + |s o (x - y)|^2) has degree 3 in each variable."""
    x, p, q = random_beam(600, seed=7, gamma=4.0)
    x = x * 1e3  # O(1) coordinates
    plan = bldtt.build_plan(x, p, n, 16, 0.9)
    assert len(plan.m2l) > 20
    st = bldtt.fmm_stages(x, p, q, plan, kernel=_poly_kernel(plan.tree.gbar))
    mass = bldtt.masses(x, p, q)
    X = torch.as_tensor(x)
    R = X[:, None, :] - X[None, :, :]
    g = _poly_kernel(plan.tree.gbar)(R, plan.tree.gbar)
    E = torch.einsum("j,ijk->ik", mass[:, 0], g)
    B = torch.linalg.cross(mass[None, :, 1:].expand_as(g), g, dim=-1).sum(1)
    tot = st["near"] + st["far"]
    np.testing.assert_allclose(tot[:, :3].numpy(), E.numpy(), rtol=1e-9, atol=1e-10 * float(E.abs().max()))
    np.testing.assert_allclose(tot[:, 3:].numpy(), B.numpy(), rtol=1e-9, atol=1e-10 * float(B.abs().max()))


def test_moments_and_m2m_identity():
    """Theorem 1 / Eq. 2.7: M2M of the children equals P2M over the parent's members."""
    x, p, q = random_beam(512, seed=5)
    plan = bldtt.build_plan(x, p, 4, 32, 0.5)
    mass = bldtt.masses(x, p, q)
    M = bldtt.upward(plan, torch.as_tensor(x), mass)
    X = torch.as_tensor(x)
    for i in (1, 2, 5, 11):
        direct = bldtt.p2m(plan, i, X, mass)
        np.testing.assert_allclose(M[i].numpy(), direct.numpy(), rtol=1e-10, atol=1e-12 * float(direct.abs().max()))
        idx = plan.tree.members[i]
        # partition of unity and linear reproduction
        np.testing.assert_allclose(M[i].sum(0).numpy(), mass[idx].sum(0).numpy(), rtol=1e-11)
        pts = plan.points(i)
        dip = (torch.as_tensor(pts).T @ M[i][:, 0]).numpy()
        np.testing.assert_allclose(dip, (X[idx].T @ mass[idx, 0]).numpy(), rtol=1e-10)


def test_cumulative_local_lemma():
    """Appendix A: L2P of the cumulative local = sum over ancestors of their own locals."""
    x, p, q = random_beam(512, seed=6)
    plan = bldtt.build_plan(x, p, 4, 32, 0.6)
    st = bldtt.fmm_stages(x, p, q, plan)
    X = torch.as_tensor(x)
    for leaf in list(plan.tree.leaves())[:4]:
        idx = plan.tree.members[leaf][:5]
        via_cum = interp.basis_3d(X[idx], plan.tree.lo[leaf], plan.tree.hi[leaf], plan.n) @ st["L"][leaf]
        direct = torch.zeros_like(via_cum)
        node = leaf
        while node >= 1:
            if node in st["Lm2l"]:
                direct = direct + interp.basis_3d(X[idx], plan.tree.lo[node], plan.tree.hi[node], plan.n) @ st["Lm2l"][node]
            node //= 2
        np.testing.assert_allclose(via_cum.numpy(), direct.numpy(), rtol=1e-9, atol=1e-11 * float(direct.abs().max()))


def test_error_falls_with_degree_and_eta():
    """Section 5 / Fig. 2: error decreases as n grows and as eta shrinks."""
    x, p, q = random_beam(1500, seed=8, gamma=10.0)
    Ed, Bd = physics.direct_fields(x, p, q)
    errs = {}
    for eta in (0.5, 0.3):
        for n in (2, 4, 6):
            E, B = bldtt.fmm_fields(x, p, q, n, 32, eta)
            errs[(eta, n)] = metrics.field_error(E.numpy(), B.numpy(), Ed.numpy(), Bd.numpy())
    for eta in (0.5, 0.3):
        assert errs[(eta, 2)] > errs[(eta, 4)] > errs[(eta, 6)]
    for n in (2, 4, 6):
        assert errs[(0.3, n)] < errs[(0.5, n)]
    assert errs[(0.5, 4)] < 1e-2


def test_single_leaf_and_tiny_inputs():
    x, p, q = random_beam(5, seed=0)
    E, B = bldtt.fmm_fields(x, p, q, 4, 8, 0.5)  # kappa = 0: one P2P(1, 1)
    Ed, Bd = physics.direct_fields(x, p, q)
    np.testing.assert_allclose(E.numpy(), Ed.numpy(), rtol=1e-13)
    E1, B1 = bldtt.fmm_fields(x[:1], p[:1], q[:1], 4, 8, 0.5)
    assert float(E1.abs().max()) == 0.0 and float(B1.abs().max()) == 0.0


def test_diam_dist_admissible_hand_values():
    """Algs. 6-8 on boxes whose half-diagonals and centre distances are known by hand."""
    s = (1.0, 1.0, 3.0)
    lo1, hi1 = np.array([0.0, 0.0, 0.0]), np.array([2.0, 4.0, 1.0])
    lo2, hi2 = np.array([10.0, 0.0, 0.0]), np.array([12.0, 4.0, 1.0])
    assert bldtt.diam(lo1, hi1, s) == np.sqrt(1.0 + 4.0 + 2.25)
    assert bldtt.dist(lo1, hi1, lo2, hi2, s) == 10.0
    assert bldtt.admissible(lo1, hi1, lo2, hi2, s, 0.27)        # sqrt(7.25)/10 = 0.269...
    assert not bldtt.admissible(lo1, hi1, lo2, hi2, s, 0.26)
    # the stretch acts on z only: separating along z by 10/3 gives the same distance
    lo3, hi3 = np.array([0.0, 0.0, 10.0 / 3.0]), np.array([2.0, 4.0, 1.0 + 10.0 / 3.0])
    assert abs(bldtt.dist(lo1, hi1, lo3, hi3, s) - 10.0) < 1e-14
    # identical boxes: d = 0 is never admissible
    assert not bldtt.admissible(lo1, hi1, lo1, hi1, s, 1e9)


@pytest.mark.parametrize("mistake", ["m2l_cross_order", "l2l_transposed", "p2p_sign", "m2m_drop_child"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    """A plausible mistake planted in the oracle makes the exactness pin fail."""
    if mistake == "m2l_cross_order":
        orig = bldtt.m2l_target

        def bad(plan, t, sources, M, kernel):
            out = orig(plan, t, sources, M, kernel)
            return torch.cat([out[:, :3], -out[:, 3:]], dim=1)
        monkeypatch.setattr(bldtt, "m2l_target", bad)
    elif mistake == "l2l_transposed":
        def bad(plan, child, parent, Lp):
            T = interp.basis_3d(torch.as_tensor(plan.points(child)), plan.tree.lo[parent],
                                plan.tree.hi[parent], plan.n)
            return T.T @ Lp
        monkeypatch.setattr(bldtt, "l2l", bad)
    elif mistake == "p2p_sign":
        orig = bldtt.p2p_target

        def bad(*a, **k):
            ti, f = orig(*a, **k)
            return ti, torch.cat([-f[:, :3], f[:, 3:]], dim=1)
        monkeypatch.setattr(bldtt, "p2p_target", bad)
    elif mistake == "m2m_drop_child":
        orig = bldtt.m2m

        def bad(plan, parent, child, Mc):
            return orig(plan, parent, child, Mc) * (0.0 if child % 2 else 1.0)
        monkeypatch.setattr(bldtt, "m2m", bad)
    with pytest.raises(AssertionError):
        test_polynomial_kernel_is_exact(3)


# ------------------------------------------------ size-aware M2L -> P2P variant
@pytest.mark.parametrize("N,N0,n,eta", [(600, 8, 2, 0.5), (1024, 16, 3, 0.5), (513, 16, 2, 0.7)])
def test_size_aware_lists_partition_all_pairs(N, N0, n, eta):
    """Substituted pairs are expanded into leaf pairs: every ordered particle
    pair is still covered once, M2L keeps only pairs with |S_t||S_s| >= m^2,
    and every admissible pair that left M2L is below m^2."""
    x, p, q = random_beam(N, seed=N + 1, gamma=20.0)
    plain = bldtt.build_plan(x, p, n, N0, eta)
    sized = bldtt.build_plan(x, p, n, N0, eta, size_aware=True)
    np.testing.assert_array_equal(_coverage(sized), np.ones((N, N), dtype=np.int64))
    tr, m2 = sized.tree, ((n + 1) ** 3) ** 2
    size = lambda i: len(tr.members[i])  # noqa: E731
    assert all(tr.is_leaf(t) and tr.is_leaf(u) for t, u in sized.p2p)
    assert all(size(t) * size(u) >= m2 for t, u in sized.m2l)
    moved = set(plain.m2l) - set(sized.m2l)
    assert moved and all(size(t) * size(u) < m2 for t, u in moved)
    assert set(sized.m2l) <= set(plain.m2l)
    assert len(sized.p2p) == len(plain.p2p) + sum(
        len(bldtt.leaves_under(tr, t)) * len(bldtt.leaves_under(tr, u)) for t, u in moved)


def test_size_aware_with_m2_above_n2_is_brute_force():
    """m^2 = 125^2 > N^2: every admissible pair is substituted, so the FMM is
    the direct sum to rounding."""
    x, p, q = random_beam(100, seed=21, gamma=5.0)
    plan = bldtt.build_plan(x, p, 4, 8, 0.5, size_aware=True)
    assert not plan.m2l and plan.p2p
    E, B = bldtt.fmm_fields(x, p, q, 4, 8, 0.5, plan=plan)
    Ed, Bd = physics.direct_fields(x, p, q)
    assert metrics.field_error(E.numpy(), B.numpy(), Ed.numpy(), Bd.numpy()) < 1e-13


def test_size_aware_error_is_not_larger():
    x, p, q = random_beam(1500, seed=22, gamma=15.0)
    Ed, Bd = physics.direct_fields(x, p, q)
    errs = []
    for sa in (False, True):
        plan = bldtt.build_plan(x, p, 2, 16, 0.5, size_aware=sa)
        E, B = bldtt.fmm_fields(x, p, q, 2, 16, 0.5, plan=plan)
        errs.append(metrics.field_error(E.numpy(), B.numpy(), Ed.numpy(), Bd.numpy()))
    assert errs[1] < errs[0], errs
