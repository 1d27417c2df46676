"""Reference gradients of the loss L = sum_i wE_i . E_i + wB_i . B_i (oracle).

Test infrastructure only; see the package docstring.

The paper has no adjoint.  Two references are kept:
* ``fmm_gradient``: the exact gradient of the FMM operator of Alg. 12 with
  its plan (tree, boxes, interaction lists, gbar) held fixed, obtained by
  automatic differentiation of ``bldtt.fmm_stages``.  This is what a
  hand-written adjoint of the FMM must reproduce to rounding.
* ``direct_gradient``: the gradient of the brute-force field (Section 5)
  with gbar held fixed, obtained the same way; the FMM gradient approaches
  it as the interpolation error vanishes.
Both are checked against central finite differences in the test-suite.

With ``gbar_term=True`` gbar is no longer a constant: it is the function
gbar(p) = sqrt(1 + pbar.pbar), pbar = (1/N) sum_j p_j, of Section 3 (below
Eq. 3.2), and dL/dp gains dL/dgbar * pbar / (N gbar) for every particle.
The tree, its boxes and the lists stay fixed (they depend on gbar only
through discrete decisions), so gbar enters the FMM only through the kernel
g of Eq. 3.2 in P2P and M2L: the interpolation points are fixed points of
the physical boxes.  The value used is the plan's gbar; only its derivative
is live.
"""
from __future__ import annotations

import torch

from . import bldtt
from .physics import as_t, direct_fields, gamma_bar, kernel_g


def _grad(fn, x, p, q, wE, wB):
    x = as_t(x).clone().requires_grad_(True)
    p = as_t(p).clone().requires_grad_(True)
    q = as_t(q).clone().requires_grad_(True)
    E, B = fn(x, p, q)
    L = (E * as_t(wE)).sum() + (B * as_t(wB)).sum()
    gx, gp, gq = torch.autograd.grad(L, (x, p, q))
    return float(L.detach()), gx.detach(), gp.detach(), gq.detach()


def live_gbar(p: torch.Tensor, value: float) -> torch.Tensor:
    """gbar(p) = sqrt(1 + pbar.pbar), pbar = (1/N) sum_j p_j (Section 3), for
    autograd: the returned scalar equals ``value`` exactly and carries the
    derivative d gbar / d p_i = pbar / (N gbar)."""
    pbar = p.mean(dim=0)
    g = torch.sqrt(1.0 + (pbar * pbar).sum())
    return value + (g - g.detach())


def fmm_gradient(x, p, q, wE, wB, plan: bldtt.Plan, gbar_term: bool = False):
    """(L, dL/dx, dL/dp, dL/dq) of the FMM with ``plan`` fixed; with
    ``gbar_term`` gbar follows p (the plan's tree, boxes and lists stay)."""
    def fn(a, b, c):
        if not gbar_term:
            return bldtt.fmm_fields(a, b, c, plan.n, plan.tree.N0, plan.eta, plan=plan)
        g = live_gbar(b, plan.tree.gbar)
        return bldtt.fmm_fields(a, b, c, plan.n, plan.tree.N0, plan.eta, plan=plan,
                                kernel=lambda R, _fixed: kernel_g(R, g))
    return _grad(fn, x, p, q, wE, wB)


def fmm_dloss_dgbar(x, p, q, wE, wB, plan: bldtt.Plan) -> float:
    """dL/dgbar of the FMM with the plan and x, p, q fixed: gbar as a leaf."""
    g = torch.tensor(float(plan.tree.gbar), dtype=torch.float64, requires_grad=True)
    E, B = bldtt.fmm_fields(x, p, q, plan.n, plan.tree.N0, plan.eta, plan=plan,
                            kernel=lambda R, _fixed: kernel_g(R, g))
    L = (E * as_t(wE)).sum() + (B * as_t(wB)).sum()
    (d,) = torch.autograd.grad(L, (g,))
    return float(d)


def direct_gradient(x, p, q, wE, wB, gbar: float | None = None, gbar_term: bool = False):
    """(L, dL/dx, dL/dp, dL/dq) of the direct sum with gbar fixed, or with
    ``gbar_term`` gbar following p (value ``gbar``, default gbar(p))."""
    if gbar is None:
        gbar = gamma_bar(as_t(p).numpy())
    if gbar_term:
        return _grad(lambda a, b, c: direct_fields(a, b, c, gbar=live_gbar(b, gbar)), x, p, q, wE, wB)
    return _grad(lambda a, b, c: direct_fields(a, b, c, gbar=gbar), x, p, q, wE, wB)


def direct_gradient_at(x, p, q, wE, wB, idx, gbar: float):
    """(dL/dx, dL/dp, dL/dq) of the direct sum for the particles ``idx`` only.

    The loss terms that depend on particle i are those of its own field (i as
    target) and those of its field at every other particle (i as source);
    autograd through exactly these terms gives the three partial derivatives
    of particle i in O(N) work, with gbar fixed.
    """
    from .physics import C0, KE, kernel_g, lorentz_gamma

    x, p, q = as_t(x), as_t(p), as_t(q)
    wE, wB = as_t(wE), as_t(wB)
    N = x.shape[0]
    a = q * lorentz_gamma(p)
    b = q[:, None] * p
    gx, gp, gq = [], [], []
    for i in [int(v) for v in idx]:
        others = torch.cat([torch.arange(0, i), torch.arange(i + 1, N)])
        xi = x[i].clone().requires_grad_(True)
        pi = p[i].clone().requires_grad_(True)
        qi = q[i].clone().requires_grad_(True)
        ai = qi * lorentz_gamma(pi[None, :])[0]
        bi = qi * pi
        g_t = kernel_g(xi[None, :] - x[others], gbar)          # i as target
        Ei = KE * (a[others][:, None] * g_t).sum(0)
        Bi = (KE / C0) * torch.linalg.cross(b[others], g_t, dim=-1).sum(0)
        g_s = kernel_g(x[others] - xi[None, :], gbar)          # i as source
        Ej = KE * ai * g_s
        Bj = (KE / C0) * torch.linalg.cross(bi[None, :].expand_as(g_s), g_s, dim=-1)
        L = (wE[i] * Ei).sum() + (wB[i] * Bi).sum() + (wE[others] * Ej).sum() + (wB[others] * Bj).sum()
        dx, dp, dq = torch.autograd.grad(L, (xi, pi, qi))
        gx.append(dx.detach())
        gp.append(dp.detach())
        gq.append(dq.detach())
    return torch.stack(gx), torch.stack(gp), torch.stack(gq)


def loss_value(E, B, wE, wB) -> float:
    return float((as_t(E) * as_t(wE)).sum() + (as_t(B) * as_t(wB)).sum())
