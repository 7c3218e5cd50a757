"""Plain FP64 CPU oracle for the convolution-quadrature (CQ) history sums and
the two-state fractional Fokker-Planck schemes of Sun, Nie & Deng,
"Fast algorithms for convolution quadrature of Riemann-Liouville fractional
derivative" (arXiv 1901.05128).

TEST INFRASTRUCTURE ONLY. Nothing in the library package may import, call or
link anything in this directory; only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it. It shares no code with the
CUDA path. It is deliberately slow and written to be checked against the
paper by eye: every function names the section / equation it follows, and
the steps run in the paper's order, vectorised over spatial DOFs only.

Modules
-------
weights     CQ weights d_{1,i} (Eq. 3.4) and d_{2,i} (Eq. 3.12).
quadrature  Gauss-Jacobi rules and the fast-form coefficients
            (Eqs. 3.6-3.7, 3.14-3.16, Remark 3.2).
history     direct history (Eq. 3.8 / 4.1) and the fast BE / SBD history
            recurrences (Eqs. 3.9-3.10, 3.17-3.18, Remarks 4.1 and 4.7).
spatial     Dirichlet finite-difference Laplacian, its eigenvalues and the
            orthonormal DST-I (the paper does not state its spatial discretisation).
scheme      BE scheme (Eq. 4.1), fast BE (Eq. 4.3), SBD scheme (Eq. 4.7) and
            fast SBD (Eq. 4.8), solved per sine mode by 2x2 Cramer's rule.
adjoint     gradients of a final-time misfit with respect to G^0 and alpha through
            the direct schemes (discrete adjoint; pinned by finite differences).

Pinning status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines, brute force or the paper's printed
properties; none is "parity unpinned".
"""
from . import weights, quadrature, history, spatial, scheme, adjoint  # noqa: F401
