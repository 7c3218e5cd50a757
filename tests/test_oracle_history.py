"""Pins of the oracle's history sums.

* direct history (Eq. 3.8 / 4.1 without i = 0) equals a brute-force strictly lower
  triangular Toeplitz matrix-vector product, which excludes G^0 (Remark 4.1);
* the fast BE / SBD recurrences (Eqs. 3.9-3.10, 3.18, Remarks 4.1 / 4.7) are geometric
  sums, so they equal a direct convolution with the quadrature weights
  (exact weights for i < 2 resp. i < Ns) up to rounding;
* against the exact weights the fast history deviates by at most sum_i |eps_i| max |G|.
"""
import numpy as np
import pytest
import scipy.linalg

import cq_inputs as ci
from oracle import history as H
from oracle import quadrature as Q
from oracle import weights as W


def _levels(n_levels, ndof, seed):
    return ci.rng(seed).standard_normal((n_levels, ndof))


@pytest.mark.parametrize("scheme", [1, 2])
def test_direct_history_is_lower_triangular_toeplitz(scheme):
    N, ndof = 57, 5
    d = W.weights(scheme, 0.4, 0.02, N)
    G = _levels(N, ndof, 11)
    col = np.concatenate([[0.0], d[1:N]])           # T[n, k] = d_{n-k} for k < n, 0 on the diagonal
    T = scipy.linalg.toeplitz(col, np.zeros(N))
    T[:, 0] = 0.0                                     # the level G^0 is not convolved
    ref = T @ G
    got = H.history_direct_all(d, G, 0, N)
    assert np.allclose(got, ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


def _quadrature_conv(d_exact, d_quad, cut, G, n):
    w = np.where(np.arange(len(d_exact)) < cut, d_exact, d_quad)
    return H.history_direct(w, G, n)


@pytest.mark.parametrize("beta,np_", [(0.3, 8), (0.75, 24)])
def test_fast_be_equals_quadrature_convolution(beta, np_):
    N, ndof, tau = 300, 7, 1.0 / 300
    G = _levels(N + 1, ndof, 3)
    fh = H.FastHistoryBE(beta, tau, np_, ndof)
    d = W.be_weights(beta, tau, N)
    dq = Q.be_quadrature_weights(beta, tau, np_, N)
    for n in range(1, N + 1):
        got = fh(n, G)
        ref = _quadrature_conv(d, dq, 2, G, n)
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * (1 + np.max(np.abs(ref)))), n


@pytest.mark.parametrize("beta,np1,np2,ns", [(0.6, 8, 12, 5), (0.3, 16, 40, 17), (0.8, 4, 4, 3)])
def test_fast_sbd_equals_quadrature_convolution(beta, np1, np2, ns):
    N, ndof, tau = 260, 6, 1.0 / 260
    G = _levels(N + 1, ndof, 5)
    fh = H.FastHistorySBD(beta, tau, np1, np2, ns, ndof)
    d = W.sbd_weights(beta, tau, N)
    dq = Q.sbd_quadrature_weights(beta, tau, np1, np2, N)
    for n in range(1, N + 1):
        got = fh(n, G)
        ref = _quadrature_conv(d, dq, ns, G, n)
        assert np.allclose(got, ref, rtol=0, atol=1e-11 * (1 + np.max(np.abs(ref)))), n


@pytest.mark.parametrize("scheme", [1, 2])
def test_fast_history_error_bound(scheme):
    beta, N, ndof, tau = 0.55, 400, 4, 1.0 / 400
    G = _levels(N + 1, ndof, 9)
    d = W.weights(scheme, beta, tau, N)
    if scheme == 1:
        fh = H.FastHistoryBE(beta, tau, 20, ndof)
        eps = np.abs(Q.be_quadrature_weights(beta, tau, 20, N) - d)
        eps[:2] = 0
    else:
        fh = H.FastHistorySBD(beta, tau, 12, 24, 15, ndof)
        eps = np.abs(Q.sbd_quadrature_weights(beta, tau, 12, 24, N) - d)
        eps[:15] = 0
    for n in range(1, N + 1):
        diff = np.max(np.abs(fh(n, G) - H.history_direct(d, G, n)))
        bound = np.sum(eps[1:n]) * np.max(np.abs(G[1:n])) if n > 1 else 0.0
        assert diff <= bound * (1 + 1e-9) + 1e-12 * abs(d[1]), n
