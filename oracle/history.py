"""Oracle: CQ history sums (test infrastructure only).

In the Fokker-Planck schemes the CQ sum at step n is sum_{i=0}^{n-1} d_i G^{n-i}
(Eqs. 4.1 and 4.7: the level G^0 is left out of the convolution, Remark 4.1).
The term d_0 G^n is implicit and handled by the time step; the explicit
*history* is

    h^n = sum_{i=1}^{n-1} d_i G^{n-i}                                  (direct)

and the fast forms replace the weights with index >= 2 (BE) or >= Ns (SBD)
by their Gauss-Jacobi sums of geometric sequences:

  fast BE (Eqs. 3.9-3.10, recurrence after Eq. 3.10, Remark 4.1)
    h^n = d_1 G^{n-1} + sum_j Ghist_j(t_n),
    Ghist_j(t_n) = r_j Ghist_j(t_{n-1}) + w_j G^{n-2}   (n >= 3; zero for n <= 2)

  fast SBD (Eq. 3.17 with the typo G(t_{n-1}) read as G(t_{n-i}), Eq. 3.18,
  recurrences after Eq. 3.18, Remark 4.7)
    h^n = sum_{i=1}^{min(Ns-1, n-1)} d_i G^{n-i} + sum_j Ghist1_j(t_n) + sum_j Ghist2_j(t_n),
    Ghist_j(t_n) = r_j Ghist_j(t_{n-1}) + q_j G^{n-Ns}   (n >= Ns+1; zero before)

Arrays of levels are indexed G[k] = G^k (shape (levels, ndof)).
"""
from __future__ import annotations

import numpy as np

from .quadrature import be_fast_coefficients, sbd_fast_coefficients
from .weights import be_weights, sbd_weights


def history_direct(d: np.ndarray, G: np.ndarray, n: int) -> np.ndarray:
    """h^n = sum_{i=1}^{n-1} d_i G^{n-i} (Eq. 3.8 / Eq. 4.1 without the i = 0 term)."""
    h = np.zeros(G.shape[1], dtype=np.float64)
    if n >= 2:
        # coefficient of level k (k = 1..n-1) is d_{n-k}
        h = d[n - 1:0:-1] @ G[1:n]
    return h


def history_direct_all(d: np.ndarray, G: np.ndarray, n_lo: int, n_hi: int) -> np.ndarray:
    """Rows h^n for n in [n_lo, n_hi), one plain sum per row."""
    return np.stack([history_direct(d, G, n) for n in range(n_lo, n_hi)]) if n_hi > n_lo else \
        np.zeros((0, G.shape[1]))


class FastHistoryBE:
    """Fast BE history parts; call with n = 1, 2, 3, ... in order."""

    def __init__(self, beta: float, tau: float, np_: int, ndof: int):
        self.d = be_weights(beta, tau, 1)
        c = be_fast_coefficients(beta, tau, np_)
        self.r, self.w = c.r, c.w
        self.parts = np.zeros((np_, ndof))
        self.n = 0

    def __call__(self, n: int, G: np.ndarray) -> np.ndarray:
        """h^n from the levels G^0..G^{n-1}; advances the history parts to t_n."""
        if n != self.n + 1:
            raise ValueError("fast history must be advanced one step at a time")
        self.n = n
        if n >= 3:
            self.parts = self.r[:, None] * self.parts + self.w[:, None] * G[n - 2][None, :]
        h = np.zeros(self.parts.shape[1])
        if n >= 2:
            h = h + self.d[1] * G[n - 1]
        return h + self.parts.sum(axis=0)


class FastHistorySBD:
    """Fast SBD history parts (two Gauss-Jacobi families); call with n = 1, 2, ... in order."""

    def __init__(self, beta: float, tau: float, np1: int, np2: int, ns: int, ndof: int):
        self.ns = ns
        self.d = sbd_weights(beta, tau, max(ns, 1))
        c = sbd_fast_coefficients(beta, tau, np1, np2, ns)
        self.r1, self.q1, self.r2, self.q2 = c.r1, c.q1, c.r2, c.q2
        self.parts1 = np.zeros((np1, ndof))
        self.parts2 = np.zeros((np2, ndof))
        self.n = 0

    def __call__(self, n: int, G: np.ndarray) -> np.ndarray:
        if n != self.n + 1:
            raise ValueError("fast history must be advanced one step at a time")
        self.n = n
        ns = self.ns
        if n - ns >= 1:
            g = G[n - ns][None, :]
            self.parts1 = self.r1[:, None] * self.parts1 + self.q1[:, None] * g
            self.parts2 = self.r2[:, None] * self.parts2 + self.q2[:, None] * g
        h = np.zeros(self.parts1.shape[1])
        for i in range(1, min(ns - 1, n - 1) + 1):
            h = h + self.d[i] * G[n - i]
        return h + self.parts1.sum(axis=0) + self.parts2.sum(axis=0)
