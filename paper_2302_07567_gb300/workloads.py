"""Seeded synthetic beams for the relativistic space-charge FMM.

This module only draws inputs: particle positions x [N,3] (metres, relative
to the bunch centre), normalised momenta p = gamma*beta [N,3] and charges
q [N] (coulomb), all float64 numpy arrays.  It holds none of the FMM's
arithmetic, so both the CUDA path and the CPU oracle may draw from it.

The paper's own workload (Section 5, Fig. 2) is a uniform cube with every
particle at gamma = 50 along z.  The other beams are the configurations the
library is measured on; where a beam description leaves a detail open the
reading chosen here is stated beside it.

Every generator uses numpy's PCG64 with the seed ``2302_07567 + tag``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2302_07567
Q_ELECTRON = -1.6e-19  # charge per macro particle in coulomb, as the beams state it
MM = 1.0e-3


@dataclass(frozen=True)
class Workload:
    """One named beam plus the FMM parameters it is run with."""

    name: str
    tag: int
    N: int
    n: int          # interpolation degree, (n+1)^3 proxy nodes per cluster
    leaf: int       # N0, maximum particles per leaf cluster
    eta: float      # admissibility parameter of the stretched condition
    passes: str     # "fwd" or "fwd+adj"
    note: str = ""
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "gauss4k": Workload(
        "gauss4k", 1, 4096, 4, 64, 0.5, "fwd",
        "Gaussian bunch sigma 1 mm, gamma 10 with 1% rms spread, 1 mrad rms angle per plane"),
    "cylinder64k": Workload(
        "cylinder64k", 2, 65536, 6, 128, 0.5, "fwd+adj",
        "uniform cylinder r 0.5 mm, length 2 mm, gamma uniform in 50 +- 5%, p along z"),
    "chirp1m": Workload(
        "chirp1m", 3, 1 << 20, 8, 256, 0.5, "fwd",
        "Gaussian 0.2/0.2/0.05 mm, linear chirp gamma 20 (tail) to 100 (head), 0.5% spread"),
    "gauss256k": Workload(
        "gauss256k", 4, 1 << 18, 6, 128, 0.5, "fwd+adj",
        "Gaussian sigma 1 mm, gamma 30 with 2% spread, p along z; Gaussian loss weights"),
    "corehalo16m": Workload(
        "corehalo16m", 5, 1 << 24, 8, 256, 0.5, "fwd+adj",
        "95% Gaussian core sigma 0.1 mm, 5% uniform shell 0.3-0.6 mm, gamma 200, 0.1% spread",
        {"recompute": True}),
    "cube": Workload(
        "cube", 6, 1_280_000, 4, 125, 0.5, "fwd",
        "the paper's Fig. 2/3 workload: uniform in [0,1]^3 m, gamma 50 along z"),
}


def _rng(tag: int, seed_offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + tag + 1000 * seed_offset))


def _p_along_z(gamma: np.ndarray) -> np.ndarray:
    p = np.zeros((gamma.size, 3))
    p[:, 2] = np.sqrt(gamma * gamma - 1.0)
    return p


def make_beam(name: str, N: int | None = None, seed_offset: int = 0):
    """Draw (x, p, q) for the named workload; ``N`` overrides the size.

    A smaller ``N`` keeps the distribution, so a sample of the workload has
    the same particle density profile and momentum spread.
    """
    w = WORKLOADS[name]
    N = w.N if N is None else int(N)
    g = _rng(w.tag, seed_offset)
    if name == "gauss4k":
        x = g.standard_normal((N, 3)) * MM
        gamma = 10.0 * (1.0 + 0.01 * g.standard_normal(N))
        th = g.standard_normal((N, 2)) * 1.0e-3
        pmag = np.sqrt(gamma * gamma - 1.0)
        norm = np.sqrt(1.0 + th[:, 0] ** 2 + th[:, 1] ** 2)
        p = np.stack([pmag * th[:, 0] / norm, pmag * th[:, 1] / norm, pmag / norm], axis=1)
    elif name == "cylinder64k":
        u = g.random(N)
        phi = g.random(N) * (2.0 * np.pi)
        r = 0.5 * MM * np.sqrt(u)
        z = (2.0 * g.random(N) - 1.0) * MM
        x = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
        gamma = 50.0 * (1.0 + 0.05 * (2.0 * g.random(N) - 1.0))
        p = _p_along_z(gamma)
    elif name == "chirp1m":
        sz = 0.05 * MM
        x = g.standard_normal((N, 3)) * np.array([0.2 * MM, 0.2 * MM, sz])
        # reading: gamma linear in z over [-3 sigma_z, +3 sigma_z], 20 at the
        # tail (-z) and 100 at the head (+z), clamped outside, then 0.5% spread
        g0 = np.clip(60.0 + 40.0 * x[:, 2] / (3.0 * sz), 20.0, 100.0)
        gamma = g0 * (1.0 + 0.005 * g.standard_normal(N))
        p = _p_along_z(gamma)
    elif name == "gauss256k":
        x = g.standard_normal((N, 3)) * MM
        gamma = 30.0 * (1.0 + 0.02 * g.standard_normal(N))
        p = _p_along_z(gamma)
    elif name == "corehalo16m":
        ncore = int(round(0.95 * N))
        nshell = N - ncore
        core = g.standard_normal((ncore, 3)) * (0.1 * MM)
        r1, r2 = 0.3 * MM, 0.6 * MM
        u = g.random(nshell)
        r = np.cbrt(r1 ** 3 + u * (r2 ** 3 - r1 ** 3))
        d = g.standard_normal((nshell, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        x = np.concatenate([core, d * r[:, None]], axis=0)
        x = x[g.permutation(N)]
        gamma = 200.0 * (1.0 + 0.001 * g.standard_normal(N))
        p = _p_along_z(gamma)
    elif name == "cube":
        x = g.random((N, 3))
        p = _p_along_z(np.full(N, 50.0))
    else:  # pragma: no cover
        raise KeyError(name)
    q = np.full(N, Q_ELECTRON)
    return np.ascontiguousarray(x), np.ascontiguousarray(p), q


def make_weights(N: int, tag: int = 4, seed_offset: int = 0):
    """Seeded loss weights (w_E, w_B), each [N,3] iid standard normal."""
    g = _rng(tag + 100, seed_offset)
    w = g.standard_normal((N, 6))
    return np.ascontiguousarray(w[:, :3]), np.ascontiguousarray(w[:, 3:])


def sample_targets(N: int, count: int, tag: int = 0) -> np.ndarray:
    """Seeded sorted subset of particle indices used for sampled error checks."""
    count = min(int(count), N)
    g = _rng(tag + 200)
    return np.sort(g.choice(N, size=count, replace=False)).astype(np.int64)


def random_beam(N: int, seed: int, gamma: float = 10.0, spread: float = 0.01,
                angle: float = 1e-3, scale=(MM, MM, MM)):
    """Small generic Gaussian beam for tests (any N, any seed)."""
    g = np.random.Generator(np.random.PCG64(SEED_BASE + 7919 * (seed + 1)))
    x = g.standard_normal((N, 3)) * np.asarray(scale, dtype=np.float64)
    gam = gamma * (1.0 + spread * g.standard_normal(N))
    th = g.standard_normal((N, 2)) * angle
    pmag = np.sqrt(np.maximum(gam * gam - 1.0, 0.0))
    norm = np.sqrt(1.0 + th[:, 0] ** 2 + th[:, 1] ** 2)
    p = np.stack([pmag * th[:, 0] / norm, pmag * th[:, 1] / norm, pmag / norm], axis=1)
    q = np.full(N, Q_ELECTRON)
    return np.ascontiguousarray(x), np.ascontiguousarray(p), q
