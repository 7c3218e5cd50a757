"""Pins of the oracle's Gauss-Jacobi rules and fast-form coefficients.

* Rules: exact moments of (1-s)^a (1+s)^b (Beta-function closed form evaluated in
  40-digit arithmetic), agreement with scipy's independent Gauss-Jacobi routine,
  and a 50-digit Newton polish of the same rule.
* BE fast weights: exact for 2 <= i <= 2 Np + 1 (Sec. 3.1 after Eq. 3.8) and not beyond.
* Integral representations Eq. 3.6 (BE) and Eq. 3.14 with Remark 3.2 (SBD) evaluated
  by adaptive high-precision quadrature reproduce the plain weights.
* SBD fast weights: the error profile eps_i shrinks with i (Remark 3.3, Figs. 1-2).
"""
import math

import mpmath
import numpy as np
import pytest
import scipy.special as sp

from oracle import quadrature as Q
from oracle import weights as W


RULES = [(1, 0.3, 0.7), (5, 0.6, 0.4), (8, 0.3, 0.7), (16, 0.6, 0.8), (31, 0.4, 1.2),
         (64, 0.2, 1.6), (128, 0.7, 0.3), (256, 0.5, 1.0)]


def _moment(a, b, k):
    # int_{-1}^{1} (1-s)^a (1+s)^b s^k ds with s = 2u - 1, u in (0,1):
    # 2^(a+b+1) sum_j C(k,j) 2^j (-1)^(k-j) B(a+1, b+j+1)
    with mpmath.workdps(60):
        a = mpmath.mpf(a)
        b = mpmath.mpf(b)
        tot = mpmath.mpf(0)
        for j in range(k + 1):
            tot += mpmath.binomial(k, j) * mpmath.mpf(2) ** j * (-1) ** (k - j) * mpmath.beta(a + 1, b + j + 1)
        return float(tot * mpmath.mpf(2) ** (a + b + 1))


@pytest.mark.parametrize("n,a,b", RULES[:5])
def test_rule_integrates_polynomials_exactly(n, a, b):
    x, lam = Q.gauss_jacobi(n, a, b)
    for k in range(2 * n):
        approx = np.sum(lam * x ** k)
        exact = _moment(a, b, k)
        scale = _moment(a, b, 0)
        assert abs(approx - exact) <= 1e-14 * scale, (k, approx, exact)


@pytest.mark.parametrize("n,a,b", RULES)
def test_rule_matches_scipy(n, a, b):
    x, lam = Q.gauss_jacobi(n, a, b)
    xs, ls = sp.roots_jacobi(n, a, b)
    assert np.max(np.abs(x - xs)) < 2e-15
    assert np.max(np.abs(lam / ls - 1.0)) < 1e-9      # scipy's tiny end weights are the looser ones
    assert abs(np.sum(lam) / (2 ** (a + b + 1) * sp.beta(a + 1, b + 1)) - 1.0) < 1e-13


@pytest.mark.parametrize("n,a,b", [(24, 0.6, 0.8), (40, 0.25, 1.5)])
def test_rule_matches_high_precision_polish(n, a, b):
    x, lam = Q.gauss_jacobi(n, a, b)
    with mpmath.workdps(50):
        A = mpmath.mpf(a)
        B = mpmath.mpf(b)
        const = (mpmath.gamma(n + A + 1) * mpmath.gamma(n + B + 1)
                 / (mpmath.gamma(n + A + B + 1) * mpmath.factorial(n)) * mpmath.mpf(2) ** (A + B + 1))
        for xj, lj in zip(x, lam):
            t = mpmath.mpf(xj)
            for _ in range(5):
                t -= mpmath.jacobi(n, A, B, t) / ((n + A + B + 1) / 2 * mpmath.jacobi(n - 1, A + 1, B + 1, t))
            dp = (n + A + B + 1) / 2 * mpmath.jacobi(n - 1, A + 1, B + 1, t)
            lw = const / ((1 - t * t) * dp * dp)
            assert abs(xj - float(t)) < 4e-16
            assert abs(lj / float(lw) - 1.0) < 1e-12


@pytest.mark.parametrize("beta", [0.2, 0.5, 0.8])
@pytest.mark.parametrize("np_", [4, 8, 16, 32])
def test_be_fast_weights_exact_up_to_2np_plus_1(beta, np_):
    tau = 1.0 / 1000.0
    n = 2 * np_ + 6
    dt = Q.be_quadrature_weights(beta, tau, np_, n)
    d = W.be_weights(beta, tau, n)
    rel = np.abs(dt / d - 1.0)
    assert np.max(rel[2:2 * np_ + 2]) < 1e-12
    if np_ <= 8:                             # larger rules converge below rounding right away
        assert rel[2 * np_ + 2] > 1e-11      # i = 2 Np + 2: the first index beyond the exactness range


@pytest.mark.parametrize("beta", [0.3, 0.7])
@pytest.mark.parametrize("i", [2, 5, 40])
def test_be_integral_representation(beta, i):
    # Eq. 3.6 evaluated by high-precision adaptive quadrature (no Gauss-Jacobi involved)
    tau = 0.01
    with mpmath.workdps(30):
        f = lambda s: (1 - s) ** beta * (1 + s) ** (1 - beta) * ((s + 1) / 2) ** (i - 2)
        integral = mpmath.quad(f, [-1, 0, 1])
        val = -integral / (4 * mpmath.mpf(tau) ** beta * mpmath.gamma(1 - beta) * mpmath.gamma(beta))
    d = W.be_weights(beta, tau, i)[i]
    assert abs(float(val) / d - 1.0) < 1e-12


@pytest.mark.parametrize("beta", [0.3, 0.6, 0.8])
@pytest.mark.parametrize("i", [3, 4, 9, 30])
def test_sbd_integral_representation_real_part(beta, i):
    # Eq. 3.14 with the real parts of Remark 3.2, evaluated by adaptive quadrature
    tau = 0.02
    with mpmath.workdps(30):
        K = 1 / (mpmath.mpf(tau) ** beta * mpmath.gamma(1 - beta) * mpmath.gamma(beta))
        wgt = lambda s: (1 - s) ** beta * (1 + s) ** (2 - 2 * beta)
        f1 = lambda s: wgt(s) * (s + 5) ** -4 * ((s + 1) / (s + 5)) ** (i - 3)
        f2 = lambda s: wgt(s) * mpmath.re(mpmath.power(mpmath.mpc(1 + 3 * s), beta)) * ((s + 1) / 2) ** (i - 3)
        I1 = mpmath.quad(f1, [-1, 1])
        I2 = mpmath.quad(f2, [-1, mpmath.mpf(-1) / 3, 1])
        val = (-mpmath.mpf(2) ** (2 + 2 * beta) * mpmath.cos(mpmath.pi * beta) * K * I1
               - mpmath.mpf(2) ** (-beta - 3) * K * I2)
    d = W.sbd_weights(beta, tau, i)[i]
    assert abs(float(val) / d - 1.0) < 1e-10


@pytest.mark.parametrize("beta", [0.3, 0.6, 0.8])
def test_sbd_fast_weights_error_profile(beta):
    tau = 1.0 / 1000.0
    n = 120
    d = W.sbd_weights(beta, tau, n)
    dt = Q.sbd_quadrature_weights(beta, tau, 31, 31, n)
    rel = np.abs(dt / d - 1.0)
    assert rel[3] > 1e-5                  # small indices are not approximated well (Remark 3.3)
    assert rel[15] < 1e-7
    assert rel[20] < 1e-9
    assert np.max(rel[60:]) < 1e-12


def test_sbd_recurrence_inputs_match_the_geometric_terms():
    beta, tau, ns = 0.45, 1.0 / 500, 17
    c = Q.sbd_fast_coefficients(beta, tau, 12, 20, ns)
    # q_j must equal w_j dbar_{Ns}(s_j): the term of index i = Ns in Eq. 3.18
    assert np.allclose(c.q1, c.w1 * (c.s1 + 5.0) ** -4 * ((c.s1 + 1) / (c.s1 + 5)) ** (ns - 3), rtol=1e-14, atol=0)
    u = 1 + 3 * c.s2
    re = np.real(np.power(u.astype(complex), beta))
    assert np.allclose(c.re13, re, rtol=1e-13, atol=0)
    assert np.allclose(c.q2, c.w2 * re * ((c.s2 + 1) / 2) ** (ns - 3), rtol=1e-13, atol=0)
