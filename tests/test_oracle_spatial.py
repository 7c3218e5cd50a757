"""Pins of the oracle's spatial operator: the DST-I is orthogonal and involutory and
diagonalises the dense finite-difference Laplacian with the stated eigenvalues."""
import numpy as np
import pytest

from oracle import spatial as S


@pytest.mark.parametrize("M", [1, 2, 7, 31])
def test_dst_is_orthogonal_involution(M):
    D = S.dst_matrix(M)
    assert np.allclose(D @ D, np.eye(M), atol=1e-13)
    assert np.allclose(D, D.T, atol=0)


@pytest.mark.parametrize("M,dim", [(5, 1), (9, 1), (3, 2), (6, 2), (2, 3), (4, 3)])
def test_dst_diagonalises_laplacian(M, dim):
    A = S.laplacian_matrix(M, dim)
    lam = S.mode_eigenvalues(M, dim)
    n = M ** dim
    basis = S.to_physical(np.eye(n), M, dim)          # row k = physical field of mode k
    for k in range(n):
        v = basis[k]
        assert np.allclose(A @ v, lam[k] * v, atol=1e-9 * lam.max())
    # coefficients of a random field reproduce it
    f = np.random.default_rng(0).standard_normal(n)
    assert np.allclose(S.to_physical(S.to_modal(f, M, dim), M, dim), f, atol=1e-13)


def test_eigenvalues_closed_form():
    M = 63
    lam = S.eigenvalues_1d(M)
    h = 1.0 / 64
    assert abs(lam[0] - np.pi ** 2) < 1e-2 * np.pi ** 2
    assert np.isclose(lam[-1], 4.0 / h ** 2 * np.sin(63 * np.pi / 128) ** 2, rtol=1e-15)


def test_3d_grid_and_mode_order():
    """3D DOFs and modes run x fastest: the mode (kz, ky, kx) = (0, 0, 1) varies along x
    only as sin(2 pi x), and its eigenvalue is lambda_1 + lambda_1 + lambda_2."""
    import cq_inputs as ci
    M = 5
    X, Y, Z = ci.grid(M, 3)
    e = np.zeros(M ** 3)
    e[1] = 1.0
    f = S.to_physical(e, M, 3)
    c = np.sqrt(2.0 / (M + 1)) ** 3
    expect = c * np.sin(np.pi * Z) * np.sin(np.pi * Y) * np.sin(2 * np.pi * X)
    assert np.allclose(f, expect, atol=1e-14)
    lam1 = S.eigenvalues_1d(M)
    assert np.isclose(S.mode_eigenvalues(M, 3)[1], 2 * lam1[0] + lam1[1], rtol=1e-15)
