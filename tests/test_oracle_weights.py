"""Pins of the oracle's CQ weights against mathematics that does not reuse its recurrences.

* BE weights (Eq. 3.4) are the scaled binomial coefficients (-1)^i C(beta, i) tau^-beta;
  their partial sums have the closed form Gamma(n+1-beta)/(Gamma(1-beta) Gamma(n+1)).
* SBD weights (Eq. 3.12): 3/2 - 2z + z^2/2 = (3/2)(1-z)(1-z/3), so the weights are
  the Cauchy product (3/2)^beta [C(beta,i)(-1)^i] * [C(beta,i)(-1)^i 3^-i] tau^-beta.
* Both: the truncated power series evaluated on |zeta| = 1/2 reproduces delta(zeta)^beta.
* CQ consistency: applied to t^mu the weights converge to the Riemann-Liouville
  derivative Gamma(mu+1)/Gamma(mu+1-beta) t^(mu-beta) at order 1 (BE) and 2 (SBD).
"""
import math

import mpmath
import numpy as np
import pytest
import scipy.special as sp

from oracle import weights as W


BETAS = [0.2, 0.3, 0.5, 0.7, 0.8]


@pytest.mark.parametrize("beta", BETAS)
def test_be_weights_are_binomial_coefficients(beta):
    tau = 1.0 / 777.0
    n = 300
    d = W.be_weights(beta, tau, n)
    i = np.arange(n + 1)
    ref = sp.binom(beta, i) * (-1.0) ** i * tau ** (-beta)
    assert np.max(np.abs(d / ref - 1.0)) < 1e-12


@pytest.mark.parametrize("beta", [0.3, 0.7])
def test_be_weight_far_index_high_precision(beta):
    n = 8192
    d = W.be_weights(beta, 1.0, n)
    with mpmath.workdps(40):
        ref = float(mpmath.binomial(beta, n) * (-1) ** n)
    assert abs(d[n] / ref - 1.0) < 1e-12


@pytest.mark.parametrize("beta", BETAS)
def test_be_partial_sums_closed_form(beta):
    n = 5000
    g = W.be_weights(beta, 1.0, n)
    S = np.cumsum(g)
    for k in (0, 1, 10, 999, 5000):
        with mpmath.workdps(40):
            ref = float(mpmath.gamma(k + 1 - beta) / (mpmath.gamma(1 - beta) * mpmath.gamma(k + 1)))
        assert abs(S[k] / ref - 1.0) < 1e-11


@pytest.mark.parametrize("beta", BETAS)
def test_sbd_weights_cauchy_product(beta):
    tau = 1.0 / 333.0
    n = 400
    d = W.sbd_weights(beta, tau, n)
    i = np.arange(n + 1)
    a = sp.binom(beta, i) * (-1.0) ** i
    b = a * 3.0 ** (-i)
    ref = np.array([np.sum(a[: k + 1][::-1] * b[: k + 1]) for k in range(n + 1)])
    ref *= 1.5 ** beta * tau ** (-beta)
    assert np.max(np.abs(d / ref - 1.0)) < 1e-12


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("beta", [0.25, 0.6, 0.9])
def test_series_reproduces_generating_function(scheme, beta):
    tau = 0.01
    n = 90
    d = W.weights(scheme, beta, tau, n)
    zeta = 0.5 * np.exp(2j * np.pi * np.arange(16) / 16)
    series = np.array([np.sum(d * z ** np.arange(n + 1)) for z in zeta])
    if scheme == 1:
        delta = (1 - zeta) / tau
    else:
        delta = ((1 - zeta) + (1 - zeta) ** 2 / 2) / tau
    exact = delta ** beta            # principal branch; Re(delta) > 0 on |zeta| = 1/2
    assert np.max(np.abs(series - exact) / np.abs(exact)) < 1e-12


@pytest.mark.parametrize("beta", BETAS)
def test_sbd_partial_sums_vanish(beta):
    # The generating function vanishes at zeta = 1, so the partial sums tend to 0 like n^-beta.
    n = 20000
    S = np.cumsum(W.sbd_weights(beta, 1.0, n))
    Sb = np.cumsum(W.be_weights(beta, 1.0, n))
    assert abs(S[n]) < 2.0 * abs(Sb[n])
    assert abs(S[n]) < abs(S[200])


def _cq_error(scheme, beta, mu, N):
    tau = 1.0 / N
    d = W.weights(scheme, beta, tau, N)
    t = np.arange(N + 1) * tau
    f = t ** mu
    approx = np.sum(d * f[::-1])          # sum_i d_i f(t_{N-i})
    exact = math.gamma(mu + 1) / math.gamma(mu + 1 - beta)
    return abs(approx - exact)


@pytest.mark.parametrize("scheme,order", [(1, 1.0), (2, 2.0)])
@pytest.mark.parametrize("beta", [0.3, 0.7])
@pytest.mark.parametrize("mu", [2, 3])
def test_cq_of_power_converges_at_scheme_order(scheme, order, beta, mu):
    errs = [_cq_error(scheme, beta, mu, N) for N in (200, 400, 800, 1600)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - order) < 0.08), rates
