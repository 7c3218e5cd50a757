"""Pins of the oracle's time stepping.

* Brute force: the whole scheme (Eq. 4.1 BE, Eq. 4.7 SBD; fast forms Eqs. 4.3 / 4.8 as
  the same schemes with the quadrature weights) assembled in physical space with the
  dense Laplacian as one block lower-triangular system and solved at once.
* Generating function of the BE solution (Eq. 4.4), inverted by FFT on a circle.
* a = 0: each state is scalar subdiffusion with the Mittag-Leffler solution
  E_alpha(-lambda t^alpha); BE converges at order 1 and the corrected SBD at order 2
  (Thms. 4.3 and 4.8).
* Fast vs direct: the difference is bounded by C n max eps_i (Thms. 4.5 / 4.10).
"""
import math

import mpmath
import numpy as np
import pytest

import cq_inputs as ci
from oracle import quadrature as Q
from oracle import scheme as SC
from oracle import spatial as SP
from oracle import weights as W


def _scheme_weights(p, beta, tau):
    """Weights the scheme convolves with: exact d_i, or for the fast forms the quadrature
    weights from index 2 (BE) / Ns (SBD) on."""
    N = p.N
    d = W.weights(p.scheme, beta, tau, N)
    if p.form == ci.DIRECT:
        return d, d
    if p.scheme == ci.BE:
        dq = Q.be_quadrature_weights(beta, tau, p.np1, N)
        cut = 2
    else:
        dq = Q.sbd_quadrature_weights(beta, tau, p.np1, p.np2, N)
        cut = p.ns
    conv = np.where(np.arange(N + 1) < cut, d, dq)
    return conv, d


def brute_force(p, G0, a=None):
    """Solve every level of the scheme at once in physical space."""
    A = SP.laplacian_matrix(p.M, p.dim)
    D = A.shape[0]
    I = np.eye(D)
    if a is None:
        a = SC.coupling(p.m)
    tau = p.T / p.N
    N = p.N
    betas = (1 - p.alpha1, 1 - p.alpha2)
    conv, exact = zip(*[_scheme_weights(p, b, tau) for b in betas])
    L = a * I + A
    K = np.zeros((2 * N * D, 2 * N * D))
    rhs = np.zeros(2 * N * D)

    def blk(n, s):
        return slice(((n - 1) * 2 + s) * D, ((n - 1) * 2 + s + 1) * D)

    def add(row, n, s, M_):          # coefficient block for level n of state s (n = 0 -> rhs)
        if n == 0:
            rhs[row] -= M_ @ G0[s]
        else:
            K[row, blk(n, s)] += M_

    for n in range(1, N + 1):
        for s in (0, 1):
            o = 1 - s
            row = blk(n, s)
            if p.scheme == ci.BE or n == 1:
                add(row, n, s, I / tau)
                add(row, n - 1, s, -I / tau)
            else:
                add(row, n, s, 1.5 * I / tau)
                add(row, n - 1, s, -2.0 * I / tau)
                add(row, n - 2, s, 0.5 * I / tau)
            if p.scheme == ci.BDF2 and n == 1:
                add(row, 1, s, 2.0 / 3.0 * conv[s][0] * L)
                add(row, 0, s, 1.0 / 3.0 * conv[s][0] * L)
                add(row, 1, o, -2.0 / 3.0 * a * conv[o][0] * I)
                add(row, 0, o, -1.0 / 3.0 * a * conv[o][0] * I)
                continue
            for i in range(0, n):
                add(row, n - i, s, conv[s][i] * L)
                add(row, n - i, o, -a * conv[o][i] * I)
            if p.scheme == ci.BDF2:
                add(row, 0, s, 0.5 * exact[s][n - 1] * L)
                add(row, 0, o, -0.5 * a * exact[o][n - 1] * I)
    X = np.linalg.solve(K, rhs)
    return X.reshape(N, 2, D)


CASES = [
    ci.Problem(0.3, 0.7, 0.4, 1.0, 9, 1, 4, ci.BE, ci.DIRECT),
    ci.Problem(0.45, 0.65, 0.7, 0.5, 8, 2, 3, ci.BE, ci.DIRECT),
    ci.Problem(0.2, 0.8, 0.3, 1.0, 10, 1, 5, ci.BDF2, ci.DIRECT),
    ci.Problem(0.6, 0.35, 0.0, 2.0, 9, 2, 2, ci.BDF2, ci.DIRECT),
    ci.Problem(0.3, 0.6, 0.6, 1.0, 12, 1, 4, ci.BE, ci.FAST, 3, 0, 2),
    ci.Problem(0.4, 0.7, 0.35, 1.0, 13, 1, 3, ci.BDF2, ci.FAST, 3, 5, 4),
    ci.Problem(0.5, 0.5, 0.8, 1.0, 11, 2, 2, ci.BDF2, ci.FAST, 2, 3, 3),
    ci.Problem(0.35, 0.75, 0.4, 1.0, 6, 3, 2, ci.BE, ci.DIRECT),         # 3D (d <= 3, Sec. 1)
    ci.Problem(0.55, 0.3, 0.65, 1.0, 5, 3, 3, ci.BDF2, ci.DIRECT),
]


@pytest.mark.parametrize("p", CASES)
def test_stepper_matches_brute_force(p):
    G0 = ci.g0_uniform(p.M, p.dim, 77)
    _, g = SC.solve(p, G0, all_levels=True)
    X = brute_force(p, G0)
    phys = np.stack([SP.to_physical(g[n], p.M, p.dim) for n in range(1, p.N + 1)])
    assert np.allclose(phys, X, rtol=0, atol=1e-12 * np.max(np.abs(X)))


def _eq44(alpha1, alpha2, a, lam, tau, zeta, g10, g20):
    """Right-hand sides of Eq. 4.4 for one mode."""
    delta = (1 - zeta) / tau
    u1 = delta ** alpha1 + a + lam
    u2 = delta ** alpha2 + a + lam
    Hz = 1.0 / (u1 * u2 - a * a)
    H1 = Hz * u2
    H2 = Hz * u1
    G1 = zeta / tau * (H1 * delta ** (alpha1 - 1) * g10 + a * Hz * delta ** (alpha1 - 1) * g20)
    G2 = zeta / tau * (a * Hz * delta ** (alpha2 - 1) * g10 + H2 * delta ** (alpha2 - 1) * g20)
    return G1, G2


@pytest.mark.parametrize("alpha1,alpha2,m,lam", [(0.3, 0.6, 0.6, 9.87), (0.7, 0.2, 0.4, 40.0), (0.5, 0.5, 0.8, 3.0)])
def test_be_solution_generating_function(alpha1, alpha2, m, lam):
    N, T = 48, 1.0
    tau = T / N
    a = SC.coupling(m)
    p = ci.Problem(alpha1, alpha2, m, T, N, 1, 1, ci.BE, ci.DIRECT)
    g0 = np.array([[0.8], [-0.3]])
    g = SC.solve_modal(p, np.array([lam]), g0)
    K = 4096
    rho = 10.0 ** (-12.0 / K)
    zeta = rho * np.exp(2j * np.pi * np.arange(K) / K)
    F1, F2 = _eq44(alpha1, alpha2, a, lam, tau, zeta, g0[0, 0], g0[1, 0])
    c1 = np.fft.fft(F1) / K / rho ** np.arange(K)        # coefficient of zeta^n
    c2 = np.fft.fft(F2) / K / rho ** np.arange(K)
    # numpy's forward FFT uses exp(-2 pi i nk/K), i.e. sum_k F(zeta_k) zeta_k^-n up to rho^n
    scale = np.max(np.abs(g))
    assert np.max(np.abs(c1[1:N + 1].real - g[1:, 0, 0])) < 1e-9 * scale
    assert np.max(np.abs(c2[1:N + 1].real - g[1:, 1, 0])) < 1e-9 * scale


def _mittag_leffler(alpha, z):
    with mpmath.workdps(60):
        z = mpmath.mpf(z)
        tot = mpmath.mpf(0)
        k = 0
        while True:
            term = z ** k / mpmath.gamma(alpha * k + 1)
            tot += term
            if k > 20 and abs(term) < mpmath.mpf(10) ** -40:
                break
            k += 1
        return float(tot)


@pytest.mark.parametrize("scheme,order", [(ci.BE, 1.0), (ci.BDF2, 2.0)])
@pytest.mark.parametrize("alpha", [0.3, 0.7])
def test_decoupled_limit_converges_to_mittag_leffler(scheme, order, alpha):
    lam = np.array([2.0])
    exact = _mittag_leffler(alpha, -2.0)          # t = 1
    errs = []
    for N in (80, 160, 320, 640):
        p = ci.Problem(alpha, alpha, 0.7, 1.0, N, 1, 1, scheme, ci.DIRECT)
        g = SC.solve_modal(p, lam, np.array([[1.0], [1.0]]), a=0.0)
        errs.append(abs(g[N, 0, 0] - exact))
        assert abs(g[N, 0, 0] - g[N, 1, 0]) < 1e-14
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - order) < 0.15), rates


@pytest.mark.parametrize("scheme", [ci.BE, ci.BDF2])
def test_fast_solution_close_to_direct(scheme):
    M, N = 15, 600
    G0 = ci.g0_nonsmooth_1d(M)
    if scheme == ci.BE:
        p = ci.Problem(0.3, 0.7, 0.6, 1.0, N, 1, M, ci.BE, ci.DIRECT, 48, 0, 2)
    else:
        p = ci.Problem(0.3, 0.7, 0.0, 1.0, N, 1, M, ci.BDF2, ci.DIRECT, 16, 48, 17)
    GD = SC.solve(p, G0)
    GF = SC.solve(p.replace(form=ci.FAST), G0)
    tau = 1.0 / N
    eps = 0.0
    for alpha in (p.alpha1, p.alpha2):
        beta = 1 - alpha
        d = W.weights(scheme, beta, tau, N)
        dq = (Q.be_quadrature_weights(beta, tau, p.np1, N) if scheme == ci.BE
              else Q.sbd_quadrature_weights(beta, tau, p.np1, p.np2, N))
        cut = 2 if scheme == ci.BE else p.ns
        eps = max(eps, np.max(np.abs(dq - d)[cut:]))
    rel = np.linalg.norm(GF - GD) / np.linalg.norm(GD)
    # Thms 4.5 / 4.10: |G_fast - G| <= C n max eps_i (|G1(0)| + |G2(0)|); the eigenvalues of A
    # enter through (a + A), so C grows with lambda_max ~ 4/h^2.
    lam_max = SP.mode_eigenvalues(M, 1).max()
    assert rel < 10 * N * eps * lam_max / np.linalg.norm(G0)
    assert rel < 1e-4
