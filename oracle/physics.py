"""Relativistic kernel, beam averages and brute-force fields (oracle, FP64).

Test infrastructure only; see the package docstring.

Section 3 of the paper (Eqs. 3.1-3.2): a source j at x_j with normalised
momentum p_j = gamma_j beta_j acts on a target at x_i with

    E_ij = q/(4 pi eps0) * gamma_j * g(x_i, x_j)
    B_ij = q/(4 pi eps0 c0) * p_j x g(x_i, x_j)
    g(x_i, x_j) = (x_i - x_j) / ((x_i-x_j)^2 + (y_i-y_j)^2 + gbar^2 (z_i-z_j)^2)^(3/2)

with gamma_j = sqrt(1 + |p_j|^2) and gbar^2 = 1 + pbar.pbar, pbar the mean
momentum of the beam.  The paper gives every particle the same charge q; a
per-particle charge q_j enters linearly and is the generalisation used here,
so the "masses" are a_j = q_j gamma_j and b_j = q_j p_j.
"""
from __future__ import annotations

import math

import numpy as np
import torch

# Reading: the paper names eps0 and c0 without values; CODATA 2018 is used.
EPS0 = 8.8541878128e-12
C0 = 299792458.0
KE = 1.0 / (4.0 * math.pi * EPS0)


def as_t(a) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.to(torch.float64)
    return torch.as_tensor(np.asarray(a, dtype=np.float64))


def lorentz_gamma(p: torch.Tensor) -> torch.Tensor:
    """gamma_j = sqrt(1 + |p_j|^2), |p|^2 summed as (px^2 + py^2) + pz^2."""
    p = as_t(p)
    return torch.sqrt(1.0 + ((p[:, 0] * p[:, 0] + p[:, 1] * p[:, 1]) + p[:, 2] * p[:, 2]))


def pairwise_sum(v) -> float:
    """Sum of a 1-D float64 array by adjacent-pair (binary-tree) summation.

    Reading: the paper averages the momentum without fixing a summation
    order.  The order used is the complete binary tree over 2^ceil(log2 N)
    terms padded with zeros: level by level, element k of the next level is
    element 2k plus element 2k+1 of the current one.  Fixing the order fixes
    gbar to the last bit, which the discrete decisions of the tree and of the
    traversal depend on.
    """
    v = np.asarray(v, dtype=np.float64).ravel()
    if v.size == 0:
        return 0.0
    L = 1
    while L < v.size:
        L *= 2
    w = np.zeros(L, dtype=np.float64)
    w[: v.size] = v
    while w.size > 1:
        w = w[0::2] + w[1::2]
    return float(w[0])


def mean_momentum(p) -> np.ndarray:
    """pbar = (1/N) sum_j p_j, each component summed by ``pairwise_sum``."""
    p = np.asarray(p, dtype=np.float64)
    N = p.shape[0]
    return np.array([pairwise_sum(p[:, k]) / N for k in range(3)])


def gamma_bar(p) -> float:
    """gbar = sqrt(1 + pbar.pbar) (Section 3, below Eq. 3.2).

    pbar.pbar is summed as (pbar_x^2 + pbar_y^2) + pbar_z^2, then 1 is added.
    """
    pb = mean_momentum(p)
    return math.sqrt(1.0 + ((pb[0] * pb[0] + pb[1] * pb[1]) + pb[2] * pb[2]))


def kernel_g(R: torch.Tensor, gbar: float) -> torch.Tensor:
    """Relativistic kernel of Eq. 3.2 for separations R = x_i - x_j [..., 3].

    Reading (the paper excludes only i == j): a separation of exactly zero
    contributes nothing, so coincident distinct particles give 0.
    """
    D = R[..., 0] * R[..., 0] + R[..., 1] * R[..., 1] + (gbar * gbar) * (R[..., 2] * R[..., 2])
    zero = D == 0
    Ds = torch.where(zero, torch.ones_like(D), D)
    inv = torch.where(zero, torch.zeros_like(D), 1.0 / (Ds * torch.sqrt(Ds)))
    return R * inv[..., None]


def _chunks(total: int, size: int):
    for s in range(0, total, size):
        yield s, min(total, s + size)


def direct_fields(x, p, q, targets=None, gbar: float | None = None, units: bool = True,
                  chunk_pairs: int = 1 << 22):
    """O(N^2) brute force of Section 5: Alg. 10 with S_t = S_s = S and i != j.

    Returns (E, B) for the rows ``targets`` (all particles by default).  With
    ``units`` the prefactors 1/(4 pi eps0) and 1/(4 pi eps0 c0) of Eq. 3.1 are
    applied.  Differentiable in x, p and q when they are tensors that
    require grad (gbar is then taken as a constant).
    """
    x, p, q = as_t(x), as_t(p), as_t(q)
    N = x.shape[0]
    if gbar is None:
        gbar = gamma_bar(p.detach().numpy())
    tgt = torch.arange(N) if targets is None else torch.as_tensor(np.asarray(targets), dtype=torch.long)
    a = q * lorentz_gamma(p)
    b = q[:, None] * p
    step = max(1, chunk_pairs // max(N, 1))
    Es, Bs = [], []
    for s, e in _chunks(tgt.numel(), step):
        ti = tgt[s:e]
        R = x[ti][:, None, :] - x[None, :, :]
        g = kernel_g(R, gbar)
        self_mask = (ti[:, None] == torch.arange(N)[None, :])
        g = torch.where(self_mask[..., None], torch.zeros_like(g), g)
        Es.append(torch.einsum("j,tjk->tk", a, g))
        Bs.append(torch.linalg.cross(b[None, :, :].expand_as(g), g, dim=-1).sum(dim=1))
    E = torch.cat(Es) if Es else torch.zeros((0, 3), dtype=torch.float64)
    B = torch.cat(Bs) if Bs else torch.zeros((0, 3), dtype=torch.float64)
    if units:
        E = E * KE
        B = B * (KE / C0)
    return E, B


def uniform_motion_fields(x, p, q, targets=None, chunk_pairs: int = 1 << 22):
    """Exact field of uniformly moving point charges (no averaging of gamma).

    E_ij = q_j gamma_j R / (4 pi eps0 (R.R + (p_j.R)^2)^(3/2)),  B_ij = beta_j x E_ij / c0,
    R = x_i - x_j: the field of a charge in uniform motion taken at its
    present position.  It equals the paper's kernel (Eq. 3.1) exactly when
    every p_j = (0, 0, p0); otherwise Eq. 3.1 is the approximation the paper
    marks with "approximately".
    """
    x, p, q = as_t(x), as_t(p), as_t(q)
    N = x.shape[0]
    tgt = torch.arange(N) if targets is None else torch.as_tensor(np.asarray(targets), dtype=torch.long)
    gam = lorentz_gamma(p)
    beta = p / gam[:, None]
    step = max(1, chunk_pairs // max(N, 1))
    Es, Bs = [], []
    for s, e in _chunks(tgt.numel(), step):
        ti = tgt[s:e]
        R = x[ti][:, None, :] - x[None, :, :]
        pr = (R * p[None, :, :]).sum(-1)
        D = (R * R).sum(-1) + pr * pr
        mask = (ti[:, None] == torch.arange(N)[None, :]) | (D == 0)
        Ds = torch.where(mask, torch.ones_like(D), D)
        inv = torch.where(mask, torch.zeros_like(D), 1.0 / (Ds * torch.sqrt(Ds)))
        Eij = (KE * q * gam)[None, :, None] * R * inv[..., None]
        Es.append(Eij.sum(1))
        Bs.append(torch.linalg.cross(beta[None].expand_as(Eij), Eij, dim=-1).sum(1) / C0)
    return torch.cat(Es), torch.cat(Bs)
