"""Oracle: convolution-quadrature weights (test infrastructure only).

d^beta_{1,i}: coefficients of ((1 - zeta)/tau)^beta               (Sec. 3.1, Eq. 3.4)
d^beta_{2,i}: coefficients of ((3/2 - 2 zeta + zeta^2/2)/tau)^beta (Sec. 3.2, Eq. 3.12)

Both are the Taylor coefficients of p(zeta)^beta for a polynomial p. With
f = p^beta one has p f' = beta p' f; equating the coefficients of zeta^(n-1)
gives, for p = p0 + p1 zeta + p2 zeta^2,

    p0 n c_n = sum_{k=1..2} ((beta+1) k - n) p_k c_{n-k},   c_0 = p0^beta,

which is the recurrence used below (for BE p = 1 - zeta and it collapses to
c_n = c_{n-1} (1 - (beta+1)/n)). The weights are c_n tau^(-beta).
"""
from __future__ import annotations

import numpy as np


def be_weights(beta: float, tau: float, n: int) -> np.ndarray:
    """d^beta_{1,i} for i = 0..n (Eq. 3.4): ((1-zeta)/tau)^beta = sum_i d_i zeta^i."""
    g = np.empty(n + 1, dtype=np.float64)
    g[0] = 1.0
    for i in range(1, n + 1):
        g[i] = g[i - 1] * (1.0 - (beta + 1.0) / i)
    return g * tau ** (-beta)


def sbd_weights(beta: float, tau: float, n: int) -> np.ndarray:
    """d^beta_{2,i} for i = 0..n (Eq. 3.12), generating function
    ((1-zeta) + (1-zeta)^2/2)/tau = (3/2 - 2 zeta + zeta^2/2)/tau."""
    p0, p1, p2 = 1.5, -2.0, 0.5
    c = np.empty(n + 1, dtype=np.float64)
    c[0] = p0 ** beta
    for k in range(1, n + 1):
        acc = ((beta + 1.0) * 1.0 - k) * p1 * c[k - 1]
        if k >= 2:
            acc += ((beta + 1.0) * 2.0 - k) * p2 * c[k - 2]
        c[k] = acc / (p0 * k)
    return c * tau ** (-beta)


def weights(scheme: int, beta: float, tau: float, n: int) -> np.ndarray:
    """Scheme 1 = BE (Eq. 3.4), scheme 2 = SBD/BDF2 (Eq. 3.12)."""
    if scheme == 1:
        return be_weights(beta, tau, n)
    if scheme == 2:
        return sbd_weights(beta, tau, n)
    raise ValueError("scheme must be 1 (BE) or 2 (BDF2)")
