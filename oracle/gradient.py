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
"""
from __future__ import annotations

import torch

from . import bldtt
from .physics import as_t, direct_fields, gamma_bar


def _grad(fn, x, p, q, wE, wB):
    x = as_t(x).clone().requires_grad_(True)
    p = as_t(p).clone().requires_grad_(True)
    q = as_t(q).clone().requires_grad_(True)
    E, B = fn(x, p, q)
    L = (E * as_t(wE)).sum() + (B * as_t(wB)).sum()
    gx, gp, gq = torch.autograd.grad(L, (x, p, q))
    return float(L.detach()), gx.detach(), gp.detach(), gq.detach()


def fmm_gradient(x, p, q, wE, wB, plan: bldtt.Plan):
    """(L, dL/dx, dL/dp, dL/dq) of the FMM with ``plan`` fixed."""
    return _grad(lambda a, b, c: bldtt.fmm_fields(a, b, c, plan.n, plan.tree.N0, plan.eta, plan=plan),
                 x, p, q, wE, wB)


def direct_gradient(x, p, q, wE, wB, gbar: float | None = None):
    """(L, dL/dx, dL/dp, dL/dq) of the direct sum with gbar fixed."""
    if gbar is None:
        gbar = gamma_bar(as_t(p).numpy())
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
