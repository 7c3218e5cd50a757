"""Oracle: spatial operator A = -Laplacian with zero Dirichlet data (test infrastructure only).

The paper leaves the spatial discretisation open (Sec. 5 gives only the mesh
size h). The workloads use the centred finite-difference Laplacian on the
M interior points per axis of (0,1)^d, h = 1/(M+1):

    (A u)_j = (2 u_j - u_{j-1} - u_{j+1}) / h^2   (per axis, summed over axes).

Its eigenvectors are the discrete sines; with the orthonormal DST-I matrix
S_{jk} = sqrt(2/(M+1)) sin(j k pi/(M+1)) (j, k = 1..M; S symmetric, S S = I)
one has A = S diag(lambda) S with lambda_k = (4/h^2) sin^2(k pi h/2) in 1D,
lambda_{k,l} = lambda_k + lambda_l in 2D and the sum over three axes in 3D (the
problem is posed for d <= 3, Sec. 1). Modes are ordered like the DOFs:
mode = ky*M + kx (2D), (kz*M + ky)*M + kx (3D).
"""
from __future__ import annotations

import numpy as np


def eigenvalues_1d(M: int) -> np.ndarray:
    h = 1.0 / (M + 1)
    k = np.arange(1, M + 1, dtype=np.float64)
    return 4.0 / h ** 2 * np.sin(k * np.pi * h / 2.0) ** 2


def mode_eigenvalues(M: int, dim: int) -> np.ndarray:
    lam = eigenvalues_1d(M)
    if dim == 1:
        return lam
    if dim == 2:
        return (lam[:, None] + lam[None, :]).reshape(-1)   # [ky, kx] -> ky*M + kx
    if dim == 3:
        return (lam[:, None, None] + lam[None, :, None] + lam[None, None, :]).reshape(-1)
    raise ValueError("dim must be 1, 2 or 3")


def dst_matrix(M: int) -> np.ndarray:
    j = np.arange(1, M + 1, dtype=np.float64)
    return np.sqrt(2.0 / (M + 1)) * np.sin(np.outer(j, j) * np.pi / (M + 1))


def to_modal(f: np.ndarray, M: int, dim: int) -> np.ndarray:
    """Sine coefficients of a field f (last axis = DOF). The transform is its own inverse."""
    S = dst_matrix(M)
    f = np.asarray(f, dtype=np.float64)
    lead = f.shape[:-1]
    if dim == 1:
        return f @ S.T
    if dim == 2:
        F = f.reshape(lead + (M, M))                    # [..., iy, ix]
        out = np.einsum("yj,...jx->...yx", S, F)        # transform along y
        out = np.einsum("...yj,xj->...yx", out, S)      # transform along x
        return out.reshape(lead + (M * M,))
    F = f.reshape(lead + (M, M, M))                     # [..., iz, iy, ix]
    out = np.einsum("zj,...jyx->...zyx", S, F)
    out = np.einsum("yj,...zjx->...zyx", S, out)
    out = np.einsum("xj,...zyj->...zyx", S, out)
    return out.reshape(lead + (M ** 3,))


to_physical = to_modal


def laplacian_matrix(M: int, dim: int) -> np.ndarray:
    """Dense FD matrix of A = -Laplacian (tests on tiny grids only)."""
    h = 1.0 / (M + 1)
    T = (2.0 * np.eye(M) - np.eye(M, k=1) - np.eye(M, k=-1)) / h ** 2
    if dim == 1:
        return T
    I = np.eye(M)
    if dim == 2:
        return np.kron(I, T) + np.kron(T, I)        # dof = iy*M + ix
    I2 = np.eye(M * M)
    return np.kron(I2, T) + np.kron(I, np.kron(T, I)) + np.kron(T, I2)   # dof = (iz*M + iy)*M + ix
