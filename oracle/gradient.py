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


def loss_value(E, B, wE, wB) -> float:
    return float((as_t(E) * as_t(wE)).sum() + (as_t(B) * as_t(wB)).sum())
