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
