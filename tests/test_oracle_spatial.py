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


@pytest.mark.parametrize("M,dim", [(5, 1), (9, 1), (3, 2), (6, 2)])
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
