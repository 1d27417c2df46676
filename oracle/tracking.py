"""Particle tracking with the FMM field (oracle, FP64; not in the paper).

Test infrastructure only; see the package docstring.

The paper's FMM (Alg. 12) evaluates the space-charge field of one particle
configuration.  A tracking code evaluates it every time step and moves the
particles with a pusher in between; the particles move little per step, so
the tree and the interaction lists of one step may serve the next.

refresh_plan keeps the tree's membership and both lists of a plan and takes
the rest from the new positions and momenta: gbar (Section 3) and every
cluster's box, the bounding box (Section 2) of its unchanged members.  The
lists still partition all N^2 particle pairs; the refreshed plan is valid
when every M2L pair is still admissible (Alg. 8) under the new boxes and
gbar, and the FMM of Alg. 12 then applies to it unchanged, with the error
bound of Section 4.

boris_push is the relativistic Boris scheme (Boris 1970, in the form of
Birdsall and Langdon, "Plasma Physics via Computer Simulation", Section
15-4) for the normalised momentum u = gamma beta:
  u-  = u + a E,                 a = q dt / (2 m c)
  t   = (a c / gamma(u-)) B,     s = 2 t / (1 + |t|^2)
  u+  = u- + (u- + u- x t) x s
  u'  = u+ + a E,                x' = x + c dt u' / gamma(u')
with gamma(u) = sqrt(1 + |u|^2).  The half kicks in E and the rotation about
B by the angle 2 atan(|t|) keep |u| in a pure magnetic field to rounding.
The operations are written in the order the CUDA kernel uses, so that both
round alike.
"""
from __future__ import annotations

import numpy as np

from .bldtt import Plan, admissible
from .physics import C0, gamma_bar
from .tree import Tree, bbox


def refresh_plan(plan: Plan, x, p):
    """(plan', valid): plan's membership and lists with gbar and boxes from (x, p)."""
    x = np.asarray(x, dtype=np.float64)
    gb = gamma_bar(np.asarray(p, dtype=np.float64))
    t = plan.tree
    C = t.C
    lo = np.zeros((C + 1, 3))
    hi = np.zeros((C + 1, 3))
    for i in range(1, C + 1):
        lo[i], hi[i] = bbox(x[t.members[i]])
    tree = Tree(t.N, t.N0, t.kappa, gb, t.members, lo, hi, t.axis)
    s = (1.0, 1.0, gb)
    valid = all(admissible(lo[i], hi[i], lo[j], hi[j], s, plan.eta) for i, j in plan.m2l)
    return Plan(tree, plan.n, plan.eta, list(plan.p2p), list(plan.m2l)), valid


def _dot(a, b):
    return (a[:, 0] * b[:, 0] + a[:, 1] * b[:, 1]) + a[:, 2] * b[:, 2]


def _cross(a, b):
    return np.stack([a[:, 1] * b[:, 2] - a[:, 2] * b[:, 1],
                     a[:, 2] * b[:, 0] - a[:, 0] * b[:, 2],
                     a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]], axis=1)


def boris_push(x, p, q, E, B, mass: float, dt: float):
    """One Boris step: returns (x', p') for fields E, B (SI) at x."""
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(p, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    a = (np.asarray(q, dtype=np.float64) * (dt / (2.0 * mass * C0)))[:, None]
    um = u + a * E
    gm = np.sqrt(1.0 + _dot(um, um))
    f = (a[:, 0] * C0) / gm
    t = f[:, None] * B
    g = 2.0 / (1.0 + _dot(t, t))
    s = g[:, None] * t
    w = um + _cross(um, t)
    up = um + _cross(w, s)
    un = up + a * E
    gn = np.sqrt(1.0 + _dot(un, un))
    v = (C0 * dt) / gn
    return x + v[:, None] * un, un
