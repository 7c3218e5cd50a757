"""Oracle: gradients of a final-time misfit through the plain (direct) schemes
(test infrastructure only).

J = 1/2 h^d sum_{s, dof} (G_s^N - Gt_s)^2 for the BE scheme (Eq. 4.1) or the SBD
scheme (Eq. 4.7). In the sine basis every mode is an independent pair x^n = (g1^n, g2^n)
with residuals (K = [[c, -a], [-a, c]], c = a + lambda, W_i = diag(d^1_i, d^2_i)):

  BE,  n >= 1:  R^n = (x^n - x^{n-1})/tau + sum_{i=0}^{n-1} K W_i x^{n-i}
  SBD, n  = 1:  R^1 = (x^1 - x^0)/tau + K W_0 (2/3 x^1 + 1/3 x^0)
  SBD, n >= 2:  R^n = (3/2 x^n - 2 x^{n-1} + 1/2 x^{n-2})/tau + sum_{i=0}^{n-1} K W_i x^{n-i} + 1/2 K W_{n-1} x^0

The Lagrangian J + sum_n (lam^n)^T R^n gives the adjoint recursion, run backwards from
m = N with mu^n = K lam^n (K is symmetric, so (K W_j)^T = W_j K):

  BE:  (I/tau + W_0 K) lam^m = -[m=N] (x^N - t) + [m<N] lam^{m+1}/tau - sum_{n>m} W_{n-m} mu^n
  SBD: (c_m I + e_m W_0 K) lam^m = -[m=N] (x^N - t) - sum_{n>m} W_{n-m} mu^n
                                   + (2/tau) lam^{m+1} - (1/(2 tau)) lam^{m+2}
       with (c_1, e_1) = (1/tau, 2/3) and (c_m, e_m) = (3/(2tau), 1) for m >= 2;

(the sum over n > m is the CQ convolution run backwards in time with the same weights),
and the gradients
  dJ/dx^0:  BE  -lam^1/tau
            SBD -lam^1/tau + 1/3 W_0 mu^1 + lam^2/(2tau) + sum_{n>=2} 1/2 W_{n-1} mu^n
  dJ/dbeta_s = sum_n mu^n_s dR^n_s/dbeta_s, i.e. the history of the solution with the
             weight derivatives d'_i = d(d_i)/d(beta) (plus the SBD first-step and G^0 terms);
  dJ/dalpha_s = -dJ/dbeta_s (beta_s = 1 - alpha_s).
The modal gradient is mapped to nodal values with the (orthonormal) sine transform.

The fast schemes (Eqs. 3.9-3.10 and 3.17-3.18 in the steppers of Remarks 4.1 and 4.7) are
the same schemes with the history weights d_i replaced, for lags i >= L (L = 2 for BE,
L = Ns for SBD), by the quadrature weights dtilde_i (Eqs. 3.8 and 3.16 without the error
term); the exact weights stay in the window i < L and in the SBD terms that carry G^0. Their
gradient (``gradient_fast``) is therefore the recursion above with dtilde in the backward
history and its beta-derivative in dJ/dbeta; the derivative of the quadrature weights is
taken by central differences of the quadrature construction, extrapolated (Richardson) from
the steps delta and delta / 2.
"""
from __future__ import annotations

import math

import numpy as np

from cq_inputs import BE, BDF2, DIRECT, FAST, Problem
from .quadrature import be_quadrature_weights, sbd_quadrature_weights
from .scheme import coupling, solve_modal
from .spatial import mode_eigenvalues, to_modal, to_physical
from .weights import weights as cq_weights


def weight_derivatives(scheme: int, beta: float, tau: float, n: int) -> np.ndarray:
    """d(d_i)/d(beta), i = 0..n, by differentiating the weight recurrences of ``oracle.weights``.

    d_i = tau^-beta c_i(beta) with c from the recurrence of Eq. 3.4 (BE) or the power-series
    recurrence of Eq. 3.12 (SBD); c'_i follows from differentiating each recurrence step.
    """
    c = np.empty(n + 1)
    dc = np.empty(n + 1)
    if scheme == BE:
        c[0], dc[0] = 1.0, 0.0
        for i in range(1, n + 1):
            f = 1.0 - (beta + 1.0) / i
            c[i] = c[i - 1] * f
            dc[i] = dc[i - 1] * f - c[i - 1] / i
    else:
        p0, p1, p2 = 1.5, -2.0, 0.5
        c[0] = p0 ** beta
        dc[0] = c[0] * math.log(p0)
        for k in range(1, n + 1):
            acc = ((beta + 1.0) - k) * p1 * c[k - 1]
            dacc = p1 * c[k - 1] + ((beta + 1.0) - k) * p1 * dc[k - 1]
            if k >= 2:
                acc += ((beta + 1.0) * 2.0 - k) * p2 * c[k - 2]
                dacc += 2.0 * p2 * c[k - 2] + ((beta + 1.0) * 2.0 - k) * p2 * dc[k - 2]
            c[k] = acc / (p0 * k)
            dc[k] = dacc / (p0 * k)
    t = tau ** (-beta)
    return t * (dc - math.log(tau) * c)


def misfit(p: Problem, GN: np.ndarray, Gt: np.ndarray) -> float:
    h = 1.0 / (p.M + 1)
    return 0.5 * h ** p.dim * float(np.sum((GN - Gt) ** 2))


def gradient(p: Problem, G0: np.ndarray, Gt: np.ndarray):
    """(J, dJ/dG0 of shape (2, M^dim), dJ/dalpha of shape (2,)) for the direct scheme of ``p``."""
    if p.form != DIRECT:
        raise ValueError("gradient covers the direct schemes; gradient_fast the fast ones")
    tau = p.T / p.N
    betas = (1.0 - p.alpha1, 1.0 - p.alpha2)
    d = [cq_weights(p.scheme, b, tau, p.N) for b in betas]
    dd = [weight_derivatives(p.scheme, b, tau, p.N) for b in betas]
    return _adjoint(p, G0, Gt, d, dd, d, dd)


def _quadrature_weights(p: Problem, beta: float, tau: float) -> np.ndarray:
    if p.scheme == BE:
        return be_quadrature_weights(beta, tau, p.np1, p.N)
    return sbd_quadrature_weights(beta, tau, p.np1, p.np2, p.N)


def gradient_fast(p: Problem, G0: np.ndarray, Gt: np.ndarray):
    """(J, dJ/dG0, dJ/dalpha) for the fast scheme of ``p``: the recursion of ``gradient`` with the
    history weights dtilde (exact below L, quadrature from L on) and their beta-derivatives."""
    if p.form != FAST:
        raise ValueError("gradient_fast covers the fast schemes")
    tau = p.T / p.N
    L = 2 if p.scheme == BE else p.ns
    betas = (1.0 - p.alpha1, 1.0 - p.alpha2)
    d = [cq_weights(p.scheme, b, tau, p.N) for b in betas]
    dd = [weight_derivatives(p.scheme, b, tau, p.N) for b in betas]
    dh, ddh = [], []
    for s, b in enumerate(betas):
        delta = min(1e-3, 0.25 * b, 0.25 * (1.0 - b))
        q = [_quadrature_weights(p, b + t, tau) for t in (delta, -delta, 0.5 * delta, -0.5 * delta)]
        dq = (4.0 * (q[2] - q[3]) / delta - (q[0] - q[1]) / (2.0 * delta)) / 3.0
        w = _quadrature_weights(p, b, tau)
        dh.append(np.where(np.arange(p.N + 1) < L, d[s], w))
        ddh.append(np.where(np.arange(p.N + 1) < L, dd[s], dq))
    return _adjoint(p, G0, Gt, dh, ddh, d, dd)


def _adjoint(p: Problem, G0: np.ndarray, Gt: np.ndarray, dh, ddh, d, dd):
    """The recursion of the module docstring for the scheme of ``p`` (direct or fast, whose
    forward levels solve_modal gives): dh / ddh are the history weights of each state and their
    beta-derivatives, d / dd the exact CQ weights and derivatives (d_0, and the SBD terms that
    carry G^0)."""
    a = coupling(p.m)
    tau = p.T / p.N
    N = p.N
    h = 1.0 / (p.M + 1)
    wd = h ** p.dim
    lam_k = mode_eigenvalues(p.M, p.dim)
    c = a + lam_k
    g0 = to_modal(G0, p.M, p.dim)
    x = solve_modal(p, lam_k, g0)                      # x[n, s, mode]
    t = to_modal(Gt, p.M, p.dim)
    r = wd * (x[N] - t)                                # dJ/dx^N
    J = 0.5 * wd * float(np.sum((x[N] - t) ** 2))

    nm = lam_k.shape[0]
    lam = np.zeros((N + 2, 2, nm))
    mu = np.zeros((N + 2, 2, nm))

    def solve_t(c0, e0, rhs):
        # (c0 I + e0 W_0 K) y = rhs, W_0 K = [[d1_0 c, -d1_0 a], [-d2_0 a, d2_0 c]]
        A11 = c0 + e0 * d[0][0] * c
        A12 = -e0 * d[0][0] * a * np.ones_like(c)
        A21 = -e0 * d[1][0] * a * np.ones_like(c)
        A22 = c0 + e0 * d[1][0] * c
        det = A11 * A22 - A12 * A21
        return np.stack([(rhs[0] * A22 - A12 * rhs[1]) / det, (A11 * rhs[1] - A21 * rhs[0]) / det])

    for m in range(N, 0, -1):
        hr = np.zeros((2, nm))
        for n in range(m + 1, N + 1):
            hr[0] += dh[0][n - m] * mu[n, 0]
            hr[1] += dh[1][n - m] * mu[n, 1]
        rhs = -hr
        if m == N:
            rhs = rhs - r
        if p.scheme == BE:
            if m < N:
                rhs = rhs + lam[m + 1] / tau
            lam[m] = solve_t(1.0 / tau, 1.0, rhs)
        else:
            if m + 1 <= N:
                rhs = rhs + 2.0 / tau * lam[m + 1]
            if m + 2 <= N:
                rhs = rhs - 0.5 / tau * lam[m + 2]
            lam[m] = solve_t(1.0 / tau, 2.0 / 3.0, rhs) if m == 1 else solve_t(1.5 / tau, 1.0, rhs)
        mu[m, 0] = c * lam[m, 0] - a * lam[m, 1]
        mu[m, 1] = -a * lam[m, 0] + c * lam[m, 1]

    # dJ/dx^0
    if p.scheme == BE:
        gx0 = -lam[1] / tau
    else:
        gx0 = -lam[1] / tau + np.stack([d[0][0] * mu[1, 0], d[1][0] * mu[1, 1]]) / 3.0
        if N >= 2:
            gx0 = gx0 + lam[2] / (2.0 * tau)
        for n in range(2, N + 1):
            gx0 = gx0 + 0.5 * np.stack([d[0][n - 1] * mu[n, 0], d[1][n - 1] * mu[n, 1]])
    # dJ/dbeta
    dbeta = np.zeros(2)
    for s in range(2):
        tot = 0.0
        for n in range(1, N + 1):
            if p.scheme == BDF2 and n == 1:
                hp = dd[s][0] * (2.0 / 3.0 * x[1, s] + 1.0 / 3.0 * x[0, s])
            else:
                hp = np.zeros(nm)
                for i in range(0, n):              # levels n-i >= 1
                    hp = hp + ddh[s][i] * x[n - i, s]
                if p.scheme == BDF2:
                    hp = hp + 0.5 * dd[s][n - 1] * x[0, s]
            tot += float(np.sum(mu[n, s] * hp))
        dbeta[s] = tot
    dG0 = to_physical(gx0, p.M, p.dim)
    return J, dG0, -dbeta
