"""Oracle: Gauss-Jacobi rules and the fast-form coefficients (test infrastructure only).

The paper only says "use the Gauss-Jacobi rule" (Sec. 3.1 after Eq. 3.8 and
Sec. 3.2 after Eq. 3.16). This oracle builds the rule for the weight
(1-s)^a (1+s)^b on [-1,1] in the textbook way:

1. Golub-Welsch: the nodes are the eigenvalues of the symmetric tridiagonal
   Jacobi matrix of the monic Jacobi polynomials (library eigen-solver as a
   step);
2. each node is polished by Newton's method on P_n^{(a,b)}, evaluated with
   the classical three-term recurrence, using
   d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)};
3. the weights come from the closed form
   lambda_j = Gamma(n+a+1) Gamma(n+b+1) / (Gamma(n+a+b+1) n!)
              * 2^(a+b+1) / ((1 - x_j^2) P_n'(x_j)^2),
   with the Gamma ratio evaluated once in 40-digit arithmetic.

Fast coefficients (the paper writes alpha for the CQ order; here beta):

BE (Eqs. 3.6-3.7): a = beta, b = 1 - beta,
    w_j = -lambda_j / (4 tau^beta Gamma(1-beta) Gamma(beta)),  r_j = (s_j + 1)/2,
    so that d_{1,i} ~ sum_j w_j r_j^(i-2) for i >= 2.

SBD (Eqs. 3.14-3.16 with Remark 3.2): a = beta, b = 2 - 2 beta, K = 1/(tau^beta Gamma(1-beta) Gamma(beta)),
    family 1: w1_j = -2^(2+2 beta) Re((-1)^(-beta)) K lambda1_j,  Re((-1)^(-beta)) = cos(pi beta),
              dbar1_i(s) = (s+5)^(-4) ((s+1)/(s+5))^(i-3);
    family 2: w2_j = -2^(-beta-3) K lambda2_j,
              dbar2_i(s) = Re((1+3s)^beta) ((s+1)/2)^(i-3),
              Re((1+3s)^beta) = |1+3s|^beta cos(pi beta) for s < -1/3;
    so that d_{2,i} ~ sum_j w1_j dbar1_i(s1_j) + sum_j w2_j dbar2_i(s2_j) for i >= 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from functools import lru_cache

import numpy as np
import scipy.linalg
import mpmath


def _jacobi_matrix(n: int, a: float, b: float):
    """Diagonal and off-diagonal of the Jacobi matrix of the monic Jacobi polynomials."""
    ab = a + b
    diag = np.empty(n)
    diag[0] = (b - a) / (ab + 2.0)
    k = np.arange(1, n, dtype=np.float64)
    diag[1:] = (b * b - a * a) / ((2 * k + ab) * (2 * k + ab + 2.0))
    off2 = 4.0 * k * (k + a) * (k + b) * (k + ab) / ((2 * k + ab) ** 2 * (2 * k + ab + 1.0) * (2 * k + ab - 1.0))
    return diag, np.sqrt(off2)


def jacobi_p(n: int, a: float, b: float, x: np.ndarray) -> np.ndarray:
    """P_n^{(a,b)}(x) by the classical three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    p1 = (a + 1.0) + (a + b + 2.0) * (x - 1.0) / 2.0
    for k in range(2, n + 1):
        c = 2.0 * k + a + b
        a1 = 2.0 * k * (k + a + b) * (c - 2.0)
        a2 = (c - 1.0) * (a * a - b * b)
        a3 = (c - 2.0) * (c - 1.0) * c
        a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c
        p0, p1 = p1, ((a2 + a3 * x) * p1 - a4 * p0) / a1
    return p1


def jacobi_dp(n: int, a: float, b: float, x: np.ndarray) -> np.ndarray:
    """d/dx P_n^{(a,b)}(x) = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}(x)."""
    if n == 0:
        return np.zeros_like(np.asarray(x, dtype=np.float64))
    return 0.5 * (n + a + b + 1.0) * jacobi_p(n - 1, a + 1.0, b + 1.0, x)


@lru_cache(maxsize=256)
def gauss_jacobi(n: int, a: float, b: float):
    """Nodes s_j (ascending) and weights lambda_j of the n-point rule for
    int_{-1}^{1} (1-s)^a (1+s)^b f(s) ds."""
    if n < 1:
        raise ValueError("n >= 1")
    diag, off = _jacobi_matrix(n, a, b)
    x = scipy.linalg.eigvalsh_tridiagonal(diag, off) if n > 1 else diag.copy()
    for _ in range(8):
        dx = jacobi_p(n, a, b, x) / jacobi_dp(n, a, b, x)
        x = x - dx
        if np.max(np.abs(dx)) < 1e-17:
            break
    with mpmath.workdps(40):
        const = mpmath.gamma(n + a + 1) * mpmath.gamma(n + b + 1) / (
            mpmath.gamma(n + a + b + 1) * mpmath.factorial(n)) * mpmath.power(2, a + b + 1)
        const = float(const)
    dp = jacobi_dp(n, a, b, x)
    lam = const / ((1.0 - x) * (1.0 + x) * dp * dp)
    x.setflags(write=False)
    lam.setflags(write=False)
    return x, lam


@dataclass(frozen=True)
class BECoeffs:
    """Fast BE rule: d_{1,i} ~ sum_j w_j r_j^(i-2), i >= 2 (Eq. 3.6-3.8)."""
    s: np.ndarray
    lam: np.ndarray
    w: np.ndarray
    r: np.ndarray


@dataclass(frozen=True)
class SBDCoeffs:
    """Fast SBD rule (Eqs. 3.14-3.16, Remark 3.2) and the recurrence inputs of
    the history parts (recurrences after Eq. 3.18):
    G_j(t_n) = r_j G_j(t_{n-1}) + q_j G(t_{n-Ns})."""
    s1: np.ndarray
    lam1: np.ndarray
    w1: np.ndarray
    r1: np.ndarray
    q1: np.ndarray
    s2: np.ndarray
    lam2: np.ndarray
    w2: np.ndarray
    r2: np.ndarray
    q2: np.ndarray
    re13: np.ndarray     # Re((1 + 3 s2_j)^beta)
    ns: int


def _gamma_product(beta: float) -> float:
    return math.gamma(1.0 - beta) * math.gamma(beta)


def be_fast_coefficients(beta: float, tau: float, np_: int) -> BECoeffs:
    """Eq. 3.6: d_{1,i} = -(4 tau^beta Gamma(1-beta) Gamma(beta))^-1
    int (1-s)^beta (1+s)^(1-beta) ((s+1)/2)^(i-2) ds, i >= 2."""
    s, lam = gauss_jacobi(np_, beta, 1.0 - beta)
    w = -lam / (4.0 * tau ** beta * _gamma_product(beta))
    r = (s + 1.0) / 2.0
    return BECoeffs(s, lam, w, r)


def re_pow_1p3s(s: np.ndarray, beta: float) -> np.ndarray:
    """Re((1+3s)^beta) with the principal branch (Remark 3.2)."""
    u = 1.0 + 3.0 * np.asarray(s, dtype=np.float64)
    return np.where(u >= 0.0, np.abs(u) ** beta, np.abs(u) ** beta * math.cos(math.pi * beta))


def sbd_fast_coefficients(beta: float, tau: float, np1: int, np2: int, ns: int) -> SBDCoeffs:
    """Eqs. 3.14-3.16 with Remark 3.2, and the history-part recurrence inputs
    q1_j = w1_j (s1_j+5)^-4 r1_j^(Ns-3), q2_j = w2_j Re((1+3 s2_j)^beta) r2_j^(Ns-3)."""
    if ns < 3:
        raise ValueError("Ns >= 3 (the integral form holds for i >= 3)")
    K = 1.0 / (tau ** beta * _gamma_product(beta))
    s1, lam1 = gauss_jacobi(np1, beta, 2.0 - 2.0 * beta)
    s2, lam2 = gauss_jacobi(np2, beta, 2.0 - 2.0 * beta)
    w1 = -(2.0 ** (2.0 + 2.0 * beta)) * math.cos(math.pi * beta) * K * lam1
    w2 = -(2.0 ** (-beta - 3.0)) * K * lam2
    r1 = (s1 + 1.0) / (s1 + 5.0)
    r2 = (s2 + 1.0) / 2.0
    re13 = re_pow_1p3s(s2, beta)
    q1 = w1 * (s1 + 5.0) ** (-4) * r1 ** (ns - 3)
    q2 = w2 * re13 * r2 ** (ns - 3)
    return SBDCoeffs(s1, lam1, w1, r1, q1, s2, lam2, w2, r2, q2, re13, ns)


def be_quadrature_weights(beta: float, tau: float, np_: int, n: int) -> np.ndarray:
    """The quadrature approximations dtilde_{1,i} = sum_j w_j r_j^(i-2), i = 0..n
    (entries i < 2 are zero: they are never approximated)."""
    c = be_fast_coefficients(beta, tau, np_)
    out = np.zeros(n + 1)
    for i in range(2, n + 1):
        out[i] = np.sum(c.w * c.r ** (i - 2))
    return out


def sbd_quadrature_weights(beta: float, tau: float, np1: int, np2: int, n: int) -> np.ndarray:
    """dtilde_{2,i} = sum_j w1_j dbar1_i(s1_j) + sum_j w2_j dbar2_i(s2_j), i = 0..n
    (Eq. 3.16 without the error term; entries i < 3 are zero)."""
    c = sbd_fast_coefficients(beta, tau, np1, np2, 3)
    out = np.zeros(n + 1)
    for i in range(3, n + 1):
        t1 = c.w1 * (c.s1 + 5.0) ** (-4) * c.r1 ** (i - 3)
        t2 = c.w2 * c.re13 * c.r2 ** (i - 3)
        out[i] = np.sum(t1) + np.sum(t2)
    return out
