"""Pins of the oracle adjoint: central finite differences of the oracle forward solve
(FP64) for dJ/dalpha and dJ/dG0, and of the weights for their beta-derivatives."""
import numpy as np
import pytest

import cq_inputs as ci
from oracle import adjoint as AD
from oracle import scheme as SC
from oracle import weights as W


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("beta", [0.3, 0.75])
def test_weight_derivatives_by_finite_differences(scheme, beta):
    tau, n, eps = 1.0 / 300, 200, 1e-6
    dd = AD.weight_derivatives(scheme, beta, tau, n)
    fd = (W.weights(scheme, beta + eps, tau, n) - W.weights(scheme, beta - eps, tau, n)) / (2 * eps)
    assert np.max(np.abs(dd - fd) / (np.abs(dd) + 1e-12 * np.max(np.abs(dd)))) < 1e-6


CASES = [ci.Problem(0.3, 0.7, 0.4, 1.0, 12, 1, 5, ci.BE, ci.DIRECT),
         ci.Problem(0.45, 0.6, 0.7, 0.5, 10, 2, 3, ci.BE, ci.DIRECT),
         ci.Problem(0.4, 0.6, 0.4, 1.0, 14, 1, 6, ci.BDF2, ci.DIRECT),
         ci.Problem(0.25, 0.8, 0.0, 1.0, 9, 2, 3, ci.BDF2, ci.DIRECT),
         ci.Problem(0.5, 0.5, 0.45, 1.0, 40, 1, 9, ci.BDF2, ci.DIRECT)]


def _J(p, G0, Gt):
    return AD.misfit(p, SC.solve(p, G0), Gt)


@pytest.mark.parametrize("p", CASES)
def test_adjoint_matches_central_differences(p):
    G0 = ci.g0_uniform(p.M, p.dim, 21)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 22)
    J, dG0, dalpha = AD.gradient(p, G0, Gt)
    assert abs(J - _J(p, G0, Gt)) <= 1e-14 * abs(J)
    eps = 1e-6
    for s, field in ((0, "alpha1"), (1, "alpha2")):
        v = getattr(p, field)
        Jp = _J(p.replace(**{field: v + eps}), G0, Gt)
        Jm = _J(p.replace(**{field: v - eps}), G0, Gt)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(dalpha[s] - fd) <= 1e-6 * abs(fd) + 1e-12, (s, dalpha[s], fd)
    rng = np.random.default_rng(3)
    for _ in range(4):
        s, k = rng.integers(2), rng.integers(G0.shape[1])
        E = np.zeros_like(G0)
        E[s, k] = 1e-5
        fd = (_J(p, G0 + E, Gt) - _J(p, G0 - E, Gt)) / 2e-5
        assert abs(dG0[s, k] - fd) <= 1e-7 * np.max(np.abs(dG0)), (s, k, dG0[s, k], fd)


FAST_CASES = [ci.Problem(0.3, 0.7, 0.4, 1.0, 30, 1, 5, ci.BE, ci.FAST, 8, 0, 2),
              ci.Problem(0.45, 0.6, 0.7, 0.5, 24, 2, 3, ci.BE, ci.FAST, 6, 0, 2),
              ci.Problem(0.4, 0.6, 0.4, 1.0, 28, 1, 6, ci.BDF2, ci.FAST, 4, 8, 5),
              ci.Problem(0.25, 0.8, 0.0, 1.0, 20, 2, 3, ci.BDF2, ci.FAST, 3, 6, 4),
              ci.Problem(0.5, 0.35, 0.45, 1.0, 4, 1, 4, ci.BDF2, ci.FAST, 3, 5, 7)]


@pytest.mark.parametrize("p", FAST_CASES)
def test_fast_adjoint_matches_central_differences(p):
    """gradient_fast against central differences of the oracle's fast forward solve (the
    quadrature tables, weights and stepper all rebuilt at alpha +- eps), and dJ/dG0 by
    differences in single coefficients of G0."""
    G0 = ci.g0_uniform(p.M, p.dim, 23)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 24)
    J, dG0, dalpha = AD.gradient_fast(p, G0, Gt)
    assert abs(J - _J(p, G0, Gt)) <= 1e-14 * abs(J)
    eps = 1e-6
    for s, field in ((0, "alpha1"), (1, "alpha2")):
        v = getattr(p, field)
        Jp = _J(p.replace(**{field: v + eps}), G0, Gt)
        Jm = _J(p.replace(**{field: v - eps}), G0, Gt)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(dalpha[s] - fd) <= 1e-6 * abs(fd) + 1e-12, (s, dalpha[s], fd)
    rng = np.random.default_rng(5)
    for _ in range(4):
        s, k = rng.integers(2), rng.integers(G0.shape[1])
        E = np.zeros_like(G0)
        E[s, k] = 1e-5
        fd = (_J(p, G0 + E, Gt) - _J(p, G0 - E, Gt)) / 2e-5
        assert abs(dG0[s, k] - fd) <= 1e-7 * np.max(np.abs(dG0)), (s, k, dG0[s, k], fd)


def test_fast_adjoint_differs_from_the_direct_one_by_the_quadrature_error():
    """The fast and direct gradients of the same problem differ by an amount of the order of the
    fast-vs-direct solution difference (Thm 4.10), not more."""
    p = ci.Problem(0.4, 0.6, 0.4, 1.0, 40, 1, 6, ci.BDF2, ci.DIRECT)
    pf = p.replace(form=ci.FAST, np1=6, np2=12, ns=6)
    G0 = ci.g0_uniform(p.M, p.dim, 25)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 26)
    _, gd, ad = AD.gradient(p, G0, Gt)
    _, gf, af = AD.gradient_fast(pf, G0, Gt)
    sol = np.max(np.abs(SC.solve(pf, G0) - SC.solve(p, G0))) / np.max(np.abs(SC.solve(p, G0)))
    assert 0.0 < np.max(np.abs(af - ad)) / np.max(np.abs(ad)) < 100 * sol + 1e-12
    assert np.max(np.abs(gf - gd)) / np.max(np.abs(gd)) < 100 * sol + 1e-12
