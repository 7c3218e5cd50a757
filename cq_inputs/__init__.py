"""Seeded synthetic inputs for the two-state fractional Fokker-Planck workloads.

This module holds only input generation: grids, initial fields and the
workload parameter sets. It contains none of the method's arithmetic (no
convolution-quadrature weights, quadrature rules, histories or time steps),
so both the CUDA path and the CPU oracle may import it.

Conventions shared by every consumer:

* domain (0,1)^d, d in {1, 2}, M interior points per axis, h = 1/(M+1),
  x_j = j*h for j = 1..M;
* a field of one state is stored DOF-contiguous with dof = iy*M + ix
  (ix fastest); a two-state field is an array of shape (2, M**d);
* random numbers come from numpy's counter-based Philox generator keyed by
  an explicit integer seed, so every machine draws the same values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import Optional

import numpy as np

SEED_BASE = 1901051280

BE = 1
BDF2 = 2
DIRECT = 0
FAST = 1


def rng(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox-4x64) keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(int(seed)))


def grid_1d(M: int) -> np.ndarray:
    """Interior grid x_j = j/(M+1), j = 1..M."""
    return np.arange(1, M + 1, dtype=np.float64) / (M + 1)


def grid(M: int, dim: int):
    """Coordinates of the interior points, flattened with dof = iy*M + ix."""
    x = grid_1d(M)
    if dim == 1:
        return (x,)
    if dim == 2:
        X = np.tile(x, M)          # ix fastest
        Y = np.repeat(x, M)
        return (X, Y)
    raise ValueError("dim must be 1 or 2")


def g0_indicator(M: int, dim: int, lo: float = 0.25, hi: float = 0.75) -> np.ndarray:
    """Both states equal to the indicator of the closed box [lo, hi]^dim."""
    pts = grid(M, dim)
    mask = np.ones(M ** dim, dtype=bool)
    for c in pts:
        mask &= (c >= lo - 1e-12) & (c <= hi + 1e-12)
    f = mask.astype(np.float64)
    return np.stack([f, f.copy()])


def g0_checkerboard_uniform(M: int, seed: int, cells: int = 8) -> np.ndarray:
    """U[0,1) values on the 'even' cells of a cells x cells checkerboard of (0,1)^2.

    A point lies on the support when floor(cells*x) + floor(cells*y) is even.
    G1 takes the first M*M draws of the stream and G2 the next M*M.
    """
    X, Y = grid(M, 2)
    support = ((np.floor(cells * X) + np.floor(cells * Y)) % 2 == 0).astype(np.float64)
    u = rng(seed).random((2, M * M))
    return u * support[None, :]


def g0_disc_gaussian(M: int, seed: int, centre=(0.5, 0.5), radius: float = 0.25) -> np.ndarray:
    """N(0,1) noise times the indicator of a closed disc (two states)."""
    X, Y = grid(M, 2)
    disc = (((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) <= radius ** 2 + 1e-12).astype(np.float64)
    z = rng(seed).standard_normal((2, M * M))
    return z * disc[None, :]


def g0_smooth_1d(M: int) -> np.ndarray:
    """Initial data (a) of Sec. 5: G1 = x(1-x), G2 = sin(x)."""
    x = grid_1d(M)
    return np.stack([x * (1.0 - x), np.sin(x)])


def g0_nonsmooth_1d(M: int) -> np.ndarray:
    """Initial data (b) of Sec. 5: G1 = (1-x) on (1/2,1), G2 = x on (0,1/2)."""
    x = grid_1d(M)
    g1 = np.where(x > 0.5, 1.0 - x, 0.0)
    g2 = np.where(x < 0.5, x, 0.0)
    return np.stack([g1, g2])


def g0_uniform(M: int, dim: int, seed: int) -> np.ndarray:
    """Plain U[0,1) field on every interior point (used by small parity cases)."""
    return rng(seed).random((2, M ** dim))


@dataclass
class Problem:
    """Parameters of one two-state fractional Fokker-Planck solve (Eqs. 1.1-1.3, 2.1).

    ``alpha1``, ``alpha2`` in (0,1); ``m`` the diagonal of the transition
    matrix; ``T`` final time; ``N`` steps (tau = T/N); ``dim``/``M`` the grid;
    ``scheme`` BE (1) or BDF2 (2); ``form`` DIRECT (0) or FAST (1);
    ``np1``, ``np2``, ``ns`` the fast-form quadrature sizes (for BE only
    ``np1`` is used and the exact window is fixed at 2).
    """
    alpha1: float
    alpha2: float
    m: float
    T: float
    N: int
    dim: int
    M: int
    scheme: int = BE
    form: int = DIRECT
    np1: int = 32
    np2: int = 32
    ns: int = 17

    @property
    def ndof(self) -> int:
        return 2 * self.M ** self.dim

    @property
    def nmodes(self) -> int:
        return self.M ** self.dim

    def replace(self, **kw) -> "Problem":
        d = asdict(self)
        d.update(kw)
        return Problem(**d)


def workload(name: str) -> tuple[Problem, np.ndarray]:
    """The named synthetic workloads: returns (problem, G0 of shape (2, M**dim)).

    * ``be1d_m63``: 1D, 63 interior points, T=1, N=1024, alpha=(0.3,0.7),
      m=0.4, BE, direct; G0 = indicator of [1/4, 3/4] on both states.
    * ``bdf2_2d_m255``: 2D 255x255, T=1, N=4096, alpha=(0.4,0.6), m=0.49,
      BDF2, fast (np1=16, np2=64, ns=17); G0 = U[0,1) on an 8x8 checkerboard,
      seed SEED_BASE+1.
    * ``grad_2d_m255``: the gradient workload: 2D 255x255, T=1, N=4096, BDF2,
      direct, alpha=(0.4,0.6), m=0.4, G0 as for ``bdf2_2d_m255``; the target is
      the same scheme's solution with alpha + (0.05, -0.05).
    * ``prec_2d_m511``: 2D 511x511, T=1, N=8192, alpha=(0.2,0.8), m=0.45,
      BE, direct (fast-form size np1 = 128); G0 = N(0,1) times the disc of
      radius 1/4 about (1/2,1/2), seed SEED_BASE+2.
    """
    if name == "be1d_m63":
        p = Problem(0.3, 0.7, 0.4, 1.0, 1024, 1, 63, BE, DIRECT, 32, 0, 2)
        return p, g0_indicator(63, 1)
    if name == "bdf2_2d_m255":
        p = Problem(0.4, 0.6, 0.49, 1.0, 4096, 2, 255, BDF2, FAST, 16, 64, 17)
        return p, g0_checkerboard_uniform(255, SEED_BASE + 1)
    if name == "grad_2d_m255":
        p = Problem(0.4, 0.6, 0.4, 1.0, 4096, 2, 255, BDF2, DIRECT, 16, 64, 17)
        return p, g0_checkerboard_uniform(255, SEED_BASE + 1)
    if name == "prec_2d_m511":
        p = Problem(0.2, 0.8, 0.45, 1.0, 8192, 2, 511, BE, DIRECT, 128, 0, 2)
        return p, g0_disc_gaussian(511, SEED_BASE + 2)
    raise KeyError(name)


def sample_indices(n_total: int, n_sample: int, seed: int) -> np.ndarray:
    """A sorted seeded sample of distinct indices in [0, n_total)."""
    n_sample = min(n_sample, n_total)
    return np.sort(rng(seed).choice(n_total, size=n_sample, replace=False))
