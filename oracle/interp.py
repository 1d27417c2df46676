"""Chebyshev interpolation points and the Lagrange basis (oracle, FP64).

Test infrastructure only; see the package docstring.

Section 2 (Eq. 2.2 and the definitions below it): a cluster S with bounding
box [a_x,b_x]x[a_y,b_y]x[a_z,b_z] carries (n+1)^3 interpolation points
xi_{S,nu} = (xi_{S,nu1}, xi_{S,nu2}, xi_{S,nu3}) and the tensor-product
Lagrange basis l_{S,nu}(x) = l^x_{nu1}(x) l^y_{nu2}(y) l^z_{nu3}(z).

Reading (the paper names no point family; its method is the barycentric
Lagrange dual tree traversal): Chebyshev points of the second kind
t_k = cos(k pi / n), k = 0..n, mapped affinely onto each side of the box,
xi_k = c + h t_k with c = (a+b)/2, h = (b-a)/2.  The oracle evaluates the
basis with the plain product formula in the normalised variable
t = (x - c)/h,

    l_k(t) = prod_{m != k} (t - t_m) / (t_k - t_m),

which is the same polynomial as in x (the affine map cancels).  Reading for a
side of zero width (b == a, all members share that coordinate): all points
coincide and the basis is l_0 = 1, l_k = 0 for k > 0.

Proxy index: nu = nu1 + (n+1) nu2 + (n+1)^2 nu3.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def cheb_points(n: int) -> np.ndarray:
    """t_k = cos(k pi / n), k = 0..n (Chebyshev points of the second kind)."""
    if n < 1:
        raise ValueError("degree n must be >= 1")
    return np.array([math.cos(k * math.pi / n) for k in range(n + 1)])


def lagrange_1d(x: torch.Tensor, a: float, b: float, n: int) -> torch.Tensor:
    """Values l_k(x), k = 0..n, of the 1-D basis on [a, b]; shape [..., n+1]."""
    x = torch.as_tensor(x, dtype=torch.float64)
    if a == b:
        out = torch.zeros(x.shape + (n + 1,), dtype=torch.float64)
        out[..., 0] = 1.0
        return out + 0.0 * x[..., None]  # keeps the graph for autograd
    c = (a + b) / 2.0
    h = (b - a) / 2.0
    t = (x - c) / h
    tk = cheb_points(n)
    cols = []
    for k in range(n + 1):
        v = torch.ones_like(t)
        for m in range(n + 1):
            if m != k:
                v = v * ((t - tk[m]) / (tk[k] - tk[m]))
        cols.append(v)
    return torch.stack(cols, dim=-1)


def points_1d(a: float, b: float, n: int) -> np.ndarray:
    """The interpolation points xi_k = c + h t_k on [a, b]."""
    if a == b:
        return np.full(n + 1, a)
    c = (a + b) / 2.0
    h = (b - a) / 2.0
    return c + h * cheb_points(n)


def proxy_points(lo, hi, n: int) -> np.ndarray:
    """All (n+1)^3 points xi_{S,nu} of a box, rows ordered by nu (x fastest)."""
    px, py, pz = (points_1d(lo[d], hi[d], n) for d in range(3))
    Z, Y, X = np.meshgrid(pz, py, px, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def basis_3d(X: torch.Tensor, lo, hi, n: int) -> torch.Tensor:
    """l_{S,nu}(x_j) for points X [P,3]; shape [P, (n+1)^3], nu x-fastest."""
    X = torch.as_tensor(X, dtype=torch.float64)
    lx = lagrange_1d(X[:, 0], float(lo[0]), float(hi[0]), n)
    ly = lagrange_1d(X[:, 1], float(lo[1]), float(hi[1]), n)
    lz = lagrange_1d(X[:, 2], float(lo[2]), float(hi[2]), n)
    P = X.shape[0]
    full = lz[:, :, None, None] * ly[:, None, :, None] * lx[:, None, None, :]
    return full.reshape(P, -1)
