"""Serial barycentric-Lagrange dual-tree-traversal FMM (oracle, FP64).

Test infrastructure only; see the package docstring.

The steps follow the paper's algorithms in their order (Alg. 12):
subdivide (Algs. 1-2) -> upward pass (Alg. 5: P2M Alg. 3 at leaves, M2M
Alg. 4 at inner nodes) -> dual tree traversal (Alg. 11, in the list-filling
form of Alg. 17) with P2P (Alg. 10) and M2L (Alg. 9) -> downward pass
(Alg. 15: L2L Alg. 13, then L2P Alg. 14 at the leaves).

Readings:
* Alg. 4 prints gamma_{S',nu'} in the momentum line; the momentum moments
  p_{S',nu'} are meant (Eq. 2.7).
* M2M, M2L and L2L accumulate (Eq. 2.7 sums over children, Eq. 2.9 adds the
  parent's cumulative local field; M2L sums over all admissible sources).
* diam and dist are those of Algs. 6-7 (half-diagonal of the stretched box
  and stretched centre distance), not the exact max/min of Eq. 4.3, as the
  paper says its implementation does.  They are evaluated with the
  operation order written below (no fused multiply-add):
  r = sqrt((v_x^2 + v_y^2) + v_z^2), v = s o ((a - b)/2), and likewise for d.
* Alg. 8 compares max(r1, r2) / d < eta literally; d = 0 gives inf or NaN
  and therefore "not admissible".
* Leaf-leaf pairs go to P2P before admissibility is tested (Algs. 11/17).
* In P2P, i == j is skipped (Section 2, after Eq. 2.6); two distinct
  particles at the same position contribute 0 (see physics.kernel_g).
* Per-particle charges: masses a_j = q_j gamma_j and b_j = q_j p_j.

A ``Plan`` holds everything that depends on positions and momenta only
through discrete decisions or constants: the tree, its boxes, gbar and the
interaction lists.  ``fmm_fields`` applied to a fixed plan is a smooth
function of (x, p, q); its autograd gradient is the gradient the adjoint
computes (tree, boxes, lists and gbar held fixed).
"""
from __future__ import annotations

import math
from collections import defaultdict
from dataclasses import dataclass, field

import numpy as np
import torch

from . import interp
from .physics import C0, KE, as_t, gamma_bar, kernel_g, lorentz_gamma
from .tree import Tree, subdivide


# --------------------------------------------------------------------- Algs. 6-8
def diam(lo, hi, s) -> float:
    """Alg. 6: || s o (a - b)/2 ||_2."""
    v = [s[k] * ((lo[k] - hi[k]) / 2.0) for k in range(3)]
    return math.sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2])


def dist(lo1, hi1, lo2, hi2, s) -> float:
    """Alg. 7: || s o (c1 - c2) ||_2 with c = (a + b)/2."""
    v = [s[k] * ((lo1[k] + hi1[k]) / 2.0 - (lo2[k] + hi2[k]) / 2.0) for k in range(3)]
    return math.sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2])


def admissible(lo1, hi1, lo2, hi2, s, eta: float) -> bool:
    """Alg. 8: max(r1, r2) / d < eta."""
    r1 = diam(lo1, hi1, s)
    r2 = diam(lo2, hi2, s)
    d = dist(lo1, hi1, lo2, hi2, s)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.float64(max(r1, r2)) / np.float64(d)
    return bool(ratio < eta)


# --------------------------------------------------------------------- Alg. 17
def leaves_under(tree: Tree, i: int) -> list:
    """The leaves of the subtree of node i (all at depth kappa)."""
    out, stack = [], [i]
    while stack:
        k = stack.pop()
        if tree.is_leaf(k):
            out.append(k)
        else:
            stack += [2 * k + 1, 2 * k]
    return sorted(out)


def dualtraverse(tree: Tree, eta: float, m2_substitute: int = 0):
    """Alg. 17 from (1, 1): returns (p2p_itl, m2l_itl) as lists of (target, source).

    With m2_substitute > 0 (the size-aware variant, not in the paper): an
    admissible pair with |S_t| |S_s| < m2_substitute is evaluated directly
    instead of by M2L, as the P2P pairs of all leaf pairs under it.  The
    particle pairs covered are the same, so the lists still partition the
    interaction matrix.
    """
    s = (1.0, 1.0, tree.gbar)
    p2p, m2l = [], []

    def rec(i: int, j: int):
        li, lj = tree.is_leaf(i), tree.is_leaf(j)
        if li and lj:
            p2p.append((i, j))
            return
        if admissible(tree.lo[i], tree.hi[i], tree.lo[j], tree.hi[j], s, eta):
            if len(tree.members[i]) * len(tree.members[j]) < m2_substitute:
                for a in leaves_under(tree, i):
                    for b in leaves_under(tree, j):
                        p2p.append((a, b))
            else:
                m2l.append((i, j))
        elif li:
            for k in (2 * j, 2 * j + 1):
                rec(i, k)
        elif lj:
            for k in (2 * i, 2 * i + 1):
                rec(k, j)
        else:
            if diam(tree.lo[i], tree.hi[i], s) > diam(tree.lo[j], tree.hi[j], s):
                for k in (2 * i, 2 * i + 1):
                    rec(k, j)
            else:
                for k in (2 * j, 2 * j + 1):
                    rec(i, k)

    rec(1, 1)
    return p2p, m2l


@dataclass
class Plan:
    tree: Tree
    n: int
    eta: float
    p2p: list
    m2l: list
    proxy: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return (self.n + 1) ** 3

    def points(self, i: int) -> np.ndarray:
        if i not in self.proxy:
            self.proxy[i] = interp.proxy_points(self.tree.lo[i], self.tree.hi[i], self.n)
        return self.proxy[i]


def build_plan(x, p, n: int, N0: int, eta: float, size_aware: bool = False) -> Plan:
    """Tree (Algs. 1-2 with s = (1,1,gbar)) plus interaction lists (Alg. 17).

    size_aware: admissible pairs with fewer particle pairs than proxy-point
    pairs, |S_t| |S_s| < m^2 with m = (n+1)^3, go to P2P instead of M2L.
    """
    x = np.asarray(x.detach().numpy() if isinstance(x, torch.Tensor) else x, dtype=np.float64)
    p = np.asarray(p.detach().numpy() if isinstance(p, torch.Tensor) else p, dtype=np.float64)
    gb = gamma_bar(p)
    tree = subdivide(x, gb, N0)
    m = (n + 1) ** 3
    p2p, m2l = dualtraverse(tree, eta, m * m if size_aware else 0)
    return Plan(tree, n, eta, p2p, m2l)


# --------------------------------------------------------------------- kernels
def _cross(b: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    return torch.linalg.cross(b.expand_as(g), g, dim=-1)


def p2m(plan: Plan, i: int, x: torch.Tensor, mass: torch.Tensor) -> torch.Tensor:
    """Alg. 3: M_{S,nu,c} = sum_j l_{S,nu}(x_j) m_{j,c}; returns [m, 4]."""
    idx = torch.as_tensor(plan.tree.members[i])
    L = interp.basis_3d(x[idx], plan.tree.lo[i], plan.tree.hi[i], plan.n)
    return L.T @ mass[idx]


def m2m(plan: Plan, parent: int, child: int, Mc: torch.Tensor) -> torch.Tensor:
    """Alg. 4 / Eq. 2.7: sum_nu' l_{S,nu}(xi_{S',nu'}) M_{S',nu'}."""
    T = interp.basis_3d(torch.as_tensor(plan.points(child)), plan.tree.lo[parent],
                        plan.tree.hi[parent], plan.n)          # [m', m]
    return T.T @ Mc


def upward(plan: Plan, x: torch.Tensor, mass: torch.Tensor) -> dict:
    """Alg. 5, post-order from the root; mass[j] = (a_j, b_j) [N, 4]."""
    M = {}

    def rec(i: int):
        if plan.tree.is_leaf(i):
            M[i] = p2m(plan, i, x, mass)
            return
        for c in (2 * i, 2 * i + 1):
            rec(c)
        acc = None
        for c in (2 * i, 2 * i + 1):
            t = m2m(plan, i, c, M[c])
            acc = t if acc is None else acc + t
        M[i] = acc

    rec(1)
    return M


def m2l_target(plan: Plan, t: int, sources, M: dict, kernel) -> torch.Tensor:
    """Alg. 9 summed over the target's sources: returns [m, 6] = (E_{t,mu}, B_{t,mu})."""
    Xt = torch.as_tensor(plan.points(t))
    Xs = torch.as_tensor(np.concatenate([plan.points(s) for s in sources]))
    Ms = torch.cat([M[s] for s in sources])                    # [k m, 4]
    g = kernel(Xt[:, None, :] - Xs[None, :, :], plan.tree.gbar)  # [m, k m, 3]
    E = torch.einsum("n,mnk->mk", Ms[:, 0], g)
    B = _cross(Ms[None, :, 1:], g).sum(1)
    return torch.cat([E, B], dim=1)


def p2p_target(plan: Plan, t: int, sources, x: torch.Tensor, mass: torch.Tensor, kernel):
    """Alg. 10 summed over the target's sources, skipping i == j."""
    ti = torch.as_tensor(plan.tree.members[t])
    sj = torch.as_tensor(np.concatenate([plan.tree.members[s] for s in sources]))
    g = kernel(x[ti][:, None, :] - x[sj][None, :, :], plan.tree.gbar)
    same = ti[:, None] == sj[None, :]
    g = torch.where(same[..., None], torch.zeros_like(g), g)
    ms = mass[sj]
    E = torch.einsum("j,tjk->tk", ms[:, 0], g)
    B = _cross(ms[None, :, 1:], g).sum(1)
    return ti, torch.cat([E, B], dim=1)


def l2l(plan: Plan, child: int, parent: int, Lp: torch.Tensor) -> torch.Tensor:
    """Alg. 13 / Eq. 2.9: sum_mu l_{S,mu}(xi_{S',mu'}) L_{S,mu}; returns [m', 6]."""
    T = interp.basis_3d(torch.as_tensor(plan.points(child)), plan.tree.lo[parent],
                        plan.tree.hi[parent], plan.n)          # [m', m]
    return T @ Lp


def l2p(plan: Plan, i: int, x: torch.Tensor, Li: torch.Tensor):
    """Alg. 14: f(x_j) += sum_mu l_{S,mu}(x_j) L_{S,mu} for the members of leaf i."""
    idx = torch.as_tensor(plan.tree.members[i])
    L = interp.basis_3d(x[idx], plan.tree.lo[i], plan.tree.hi[i], plan.n)
    return idx, L @ Li


def downward(plan: Plan, Lm2l: dict, x: torch.Tensor):
    """Alg. 15, pre-order: cumulative local fields, then L2P at the leaves."""
    m = plan.m
    zero = torch.zeros((m, 6), dtype=torch.float64)
    cum = {1: Lm2l.get(1, zero)}
    rows, vals = [], []

    def rec(i: int):
        if plan.tree.is_leaf(i):
            idx, f = l2p(plan, i, x, cum[i])
            rows.append(idx)
            vals.append(f)
            return
        for c in (2 * i, 2 * i + 1):
            cum[c] = Lm2l.get(c, zero) + l2l(plan, c, i, cum[i])
        for c in (2 * i, 2 * i + 1):
            rec(c)

    rec(1)
    return cum, rows, vals


def masses(x, p, q):
    x, p, q = as_t(x), as_t(p), as_t(q)
    a = q * lorentz_gamma(p)
    b = q[:, None] * p
    return torch.cat([a[:, None], b], dim=1)


def fmm_stages(x, p, q, plan: Plan, kernel=kernel_g):
    """Alg. 12 on a given plan; returns a dict with every intermediate.

    Keys: M (node -> [m,4] multipoles), L (node -> [m,6] cumulative locals),
    near/far ([N,6] unscaled (E,B) parts), E and B ([N,3], with the
    prefactors of Eq. 3.1 applied).
    """
    x, p, q = as_t(x), as_t(p), as_t(q)
    N = x.shape[0]
    mass = masses(x, p, q)
    M = upward(plan, x, mass)

    by_t = defaultdict(list)
    for t, s in plan.m2l:
        by_t[t].append(s)
    Lm2l = {t: m2l_target(plan, t, srcs, M, kernel) for t, srcs in sorted(by_t.items())}

    by_t = defaultdict(list)
    for t, s in plan.p2p:
        by_t[t].append(s)
    near = torch.zeros((N, 6), dtype=torch.float64)
    for t, srcs in sorted(by_t.items()):
        ti, f = p2p_target(plan, t, srcs, x, mass, kernel)
        near = near.index_add(0, ti, f)

    cum, rows, vals = downward(plan, Lm2l, x)
    far = torch.zeros((N, 6), dtype=torch.float64)
    for idx, f in zip(rows, vals):
        far = far.index_add(0, idx, f)
    tot = near + far
    return dict(M=M, L=cum, Lm2l=Lm2l, near=near, far=far,
                E=tot[:, :3] * KE, B=tot[:, 3:] * (KE / C0))


def fmm_fields(x, p, q, n: int, N0: int, eta: float, plan: Plan | None = None, kernel=kernel_g):
    """E, B [N,3] of the FMM (Alg. 12); builds the plan from (x, p) if not given."""
    if plan is None:
        plan = build_plan(x, p, n, N0, eta)
    st = fmm_stages(x, p, q, plan, kernel)
    return st["E"], st["B"]
