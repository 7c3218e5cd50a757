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
    """Coordinates of the interior points, flattened with dof = iy*M + ix (2D) or
    (iz*M + iy)*M + ix (3D)."""
    x = grid_1d(M)
    if dim == 1:
        return (x,)
    if dim == 2:
        X = np.tile(x, M)          # ix fastest
        Y = np.repeat(x, M)
        return (X, Y)
    if dim == 3:
        X = np.tile(x, M * M)
        Y = np.tile(np.repeat(x, M), M)
        Z = np.repeat(x, M * M)
        return (X, Y, Z)
    raise ValueError("dim must be 1, 2 or 3")


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


def lowest_eigenvalue(M: int, dim: int) -> float:
    """Smallest eigenvalue of the centred FD Dirichlet Laplacian on (0,1)^dim (M points per axis)."""
    h = 1.0 / (M + 1)
    return dim * 4.0 / h ** 2 * math.sin(math.pi * h / 2.0) ** 2


def growth_rate(alpha1: float, alpha2: float, m: float, lam: float) -> float:
    """Largest real z > 0 with (z^a1 + a + lam)(z^a2 + a + lam) = a^2, a = (1-m)/(2m-1):
    the growth rate of the mode with eigenvalue lam of the continuous problem (a pole of
    H(z) in Eq. 2.2); 0 when there is none. Used only to screen random problem draws."""
    a = (1.0 - m) / (2.0 * m - 1.0)
    c = a + lam
    f = lambda z: (z ** alpha1 + c) * (z ** alpha2 + c) - a * a
    if f(0.0) >= 0.0:                      # both factors keep their sign: no positive root
        return 0.0
    lo, hi = 0.0, 1.0
    while f(hi) < 0.0:
        hi *= 2.0
        if hi > 1e300:
            return math.inf
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return hi


def batch_workload(n: int = 256, seed: int = SEED_BASE + 4, growth_limit: float = 600.0):
    """Independent instances of uneven parameters (fast FP64 form), drawn from one seeded stream:
    alpha_i ~ U(0.1, 0.9); m ~ U([0.30, 0.48]) or U([0.52, 0.70]) (50/50); 1D with M log-uniform
    in [31, 1023] or 2D with M log-uniform in [31, 255] (50/50); N log-uniform in [512, 8192];
    BE or BDF2 (50/50); T = 1. Fast sizes: BE Np = 64 (N <= 2048) or 128; BDF2 Np1 = 16,
    Np2 = 64 (N <= 4096) or 96, Ns = 17. A draw whose lowest mode grows faster than
    growth_limit / T (see growth_rate) is replaced by the next draw; the number of
    replaced draws is returned. G0 = U[0,1) on the closed box [1/4, 3/4]^dim, both states.
    Returns (problems, G0 list, redraws)."""
    r = rng(seed)
    probs, fields, redraws = [], [], 0
    while len(probs) < n:
        a1, a2 = r.uniform(0.1, 0.9, 2)
        m = r.uniform(0.30, 0.48) if r.random() < 0.5 else r.uniform(0.52, 0.70)
        dim = 1 if r.random() < 0.5 else 2
        Mmax = 1023 if dim == 1 else 255
        M = int(round(math.exp(r.uniform(math.log(31), math.log(Mmax)))))
        N = int(round(math.exp(r.uniform(math.log(512), math.log(8192)))))
        scheme = BE if r.random() < 0.5 else BDF2
        if growth_rate(a1, a2, m, lowest_eigenvalue(M, dim)) * 1.0 > growth_limit:
            redraws += 1
            continue
        if scheme == BE:
            p = Problem(float(a1), float(a2), float(m), 1.0, N, dim, M, BE, FAST, 64 if N <= 2048 else 128, 0, 2)
        else:
            p = Problem(float(a1), float(a2), float(m), 1.0, N, dim, M, BDF2, FAST, 16, 64 if N <= 4096 else 96, 17)
        pts = grid(M, dim)
        box = np.ones(M ** dim, dtype=bool)
        for c in pts:
            box &= (c >= 0.25 - 1e-12) & (c <= 0.75 + 1e-12)
        fields.append(r.random((2, M ** dim)) * box[None, :])
        probs.append(p)
    return probs, fields, redraws


def sample_indices(n_total: int, n_sample: int, seed: int) -> np.ndarray:
    """A sorted seeded sample of distinct indices in [0, n_total)."""
    n_sample = min(n_sample, n_total)
    return np.sort(rng(seed).choice(n_total, size=n_sample, replace=False))
