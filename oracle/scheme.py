"""Oracle: time stepping of the two-state fractional Fokker-Planck system (test infrastructure only).

System (Eq. 2.1), with a = (1-m)/(2m-1) and beta_i = 1 - alpha_i the CQ orders:
    dG1/dt + a D^{beta1} G1 + D^{beta1} A G1 = a D^{beta2} G2,   and symmetrically for G2.

In the sine basis A is diagonal, so every mode k (eigenvalue lambda_k) gives
an independent pair (g1, g2). Writing c = a + lambda_k, d^s the weights of
state s and h_s^n its history (``oracle.history``):

BE scheme, n >= 1 (Eq. 4.1; fast BE Eq. 4.3 uses the fast history):
    (1/tau + c d^1_0) g1^n - a d^2_0 g2^n = g1^{n-1}/tau - c h1^n + a h2^n
    -a d^1_0 g1^n + (1/tau + c d^2_0) g2^n = g2^{n-1}/tau - c h2^n + a h1^n

SBD scheme (Eq. 4.7; fast SBD Eq. 4.8 uses the fast history, Remark 4.7):
  n = 1 (the corrected first step):
    (1/tau + 2/3 c d^1_0) g1^1 - 2/3 a d^2_0 g2^1 = g1^0/tau - 1/3 c d^1_0 g1^0 + 1/3 a d^2_0 g2^0
    and symmetrically;
  n >= 2:
    (3/(2tau) + c d^1_0) g1^n - a d^2_0 g2^n
        = (2 g1^{n-1} - g1^{n-2}/2)/tau - c (h1^n + d^1_{n-1} g1^0/2) + a (h2^n + d^2_{n-1} g2^0/2)
    and symmetrically. The weight d_{n-1} of the G^0 correction is the exact
    CQ weight in both the plain and the fast scheme.

Each 2x2 system is solved by Cramer's rule.
"""
from __future__ import annotations

import numpy as np

from cq_inputs import Problem, BE, BDF2, DIRECT, FAST
from .weights import weights as cq_weights
from .history import history_direct, FastHistoryBE, FastHistorySBD
from .spatial import mode_eigenvalues, to_modal, to_physical


class SingularStep(ArithmeticError):
    pass


def coupling(m: float) -> float:
    """a = (1 - m)/(2m - 1) (Sec. 2, after Eq. 2.1)."""
    return (1.0 - m) / (2.0 * m - 1.0)


def _solve2(A11, A12, A21, A22, b1, b2):
    det = A11 * A22 - A12 * A21
    scale = np.maximum(np.abs(A11 * A22), np.abs(A12 * A21))
    if np.any(np.abs(det) <= 1e-14 * scale):
        raise SingularStep("2x2 step matrix is singular to working precision")
    return (b1 * A22 - A12 * b2) / det, (A11 * b2 - A21 * b1) / det


def _histories(p: Problem, betas, tau, nm):
    if p.form == DIRECT:
        return None
    if p.scheme == BE:
        return [FastHistoryBE(b, tau, p.np1, nm) for b in betas]
    return [FastHistorySBD(b, tau, p.np1, p.np2, p.ns, nm) for b in betas]


def solve_modal(p: Problem, lam: np.ndarray, g0: np.ndarray, a: float | None = None) -> np.ndarray:
    """All modal levels g[n, s, mode], n = 0..N, of the scheme chosen by ``p``.

    ``a`` overrides the coupling a(m) (tests only, e.g. a = 0 decouples the states).
    """
    if a is None:
        a = coupling(p.m)
    tau = p.T / p.N
    betas = (1.0 - p.alpha1, 1.0 - p.alpha2)
    N = p.N
    nm = lam.shape[0]
    d = [cq_weights(p.scheme, b, tau, N) for b in betas]
    fast = _histories(p, betas, tau, nm)
    g = np.zeros((N + 1, 2, nm))
    g[0] = g0
    c = a + lam
    for n in range(1, N + 1):
        if fast is None:
            h1 = history_direct(d[0], g[:, 0], n)
            h2 = history_direct(d[1], g[:, 1], n)
        else:
            h1 = fast[0](n, g[:, 0])
            h2 = fast[1](n, g[:, 1])
        d10, d20 = d[0][0], d[1][0]
        if p.scheme == BE:
            A11 = 1.0 / tau + c * d10
            A22 = 1.0 / tau + c * d20
            A12 = -a * d20 * np.ones_like(c)
            A21 = -a * d10 * np.ones_like(c)
            b1 = g[n - 1, 0] / tau - c * h1 + a * h2
            b2 = g[n - 1, 1] / tau - c * h2 + a * h1
        elif n == 1:
            A11 = 1.0 / tau + 2.0 / 3.0 * c * d10
            A22 = 1.0 / tau + 2.0 / 3.0 * c * d20
            A12 = -2.0 / 3.0 * a * d20 * np.ones_like(c)
            A21 = -2.0 / 3.0 * a * d10 * np.ones_like(c)
            b1 = g[0, 0] / tau - c * d10 * g[0, 0] / 3.0 + a * d20 * g[0, 1] / 3.0
            b2 = g[0, 1] / tau - c * d20 * g[0, 1] / 3.0 + a * d10 * g[0, 0] / 3.0
        else:
            A11 = 1.5 / tau + c * d10
            A22 = 1.5 / tau + c * d20
            A12 = -a * d20 * np.ones_like(c)
            A21 = -a * d10 * np.ones_like(c)
            e1 = h1 + 0.5 * d[0][n - 1] * g[0, 0]
            e2 = h2 + 0.5 * d[1][n - 1] * g[0, 1]
            b1 = (2.0 * g[n - 1, 0] - 0.5 * g[n - 2, 0]) / tau - c * e1 + a * e2
            b2 = (2.0 * g[n - 1, 1] - 0.5 * g[n - 2, 1]) / tau - c * e2 + a * e1
        g[n, 0], g[n, 1] = _solve2(A11, A12, A21, A22, b1, b2)
    return g


def solve(p: Problem, G0: np.ndarray, a: float | None = None, all_levels: bool = False):
    """Physical G^N (shape (2, M**dim)) from physical G^0; optionally all modal levels too."""
    lam = mode_eigenvalues(p.M, p.dim)
    g0 = to_modal(G0, p.M, p.dim)
    g = solve_modal(p, lam, g0, a=a)
    GN = to_physical(g[p.N], p.M, p.dim)
    return (GN, g) if all_levels else GN
