"""GPU gradient (fp2s_gradient, discrete adjoint of the direct schemes) against the
oracle's FP64 adjoint and against central finite differences of the GPU forward solve
(``-m gpu``).

Tolerances: J to 1e-12 relative (same forward arithmetic as the parity tests); the
gradients are sums over modes and steps of adjoint-weighted terms whose rounding
differs between the two sides, so dJ/dalpha is compared at 1e-9 relative and dJ/dG0
at 1e-10 of its largest entry. Finite differences (step 1e-5, FP64) are accurate to
~1e-9 relative here; the bar is 1e-6 relative.
"""
import numpy as np
import pytest

import cq_inputs as ci
from oracle import adjoint as AD

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_05128_gb300 as pkg
    pkg.build()
    return pkg.load()


def _cp(fc, p, prec=0):
    return fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, ci.DIRECT, prec=prec)


def _grad(fc, p, G0, Gt, prec=0):
    cp = _cp(fc, p, prec)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gt = torch.tensor(Gt, dtype=torch.float64, device="cuda")
    dg = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_gradient(cp, g0, gt, dg, None), "cuda")
    J, da = fc.fp2s_gradient(cp, g0, gt, dg, ws)
    return J, dg.cpu().numpy(), np.array(da)


def _J_gpu(fc, p, G0, Gt, prec=0):
    cp = _cp(fc, p, prec)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), "cuda")
    fc.fp2s_solve(cp, g0, gN, ws)
    GN = gN.cpu().numpy()
    h = 1.0 / (p.M + 1)
    return 0.5 * h ** p.dim * float(np.sum((GN - Gt) ** 2))


CASES = [ci.Problem(0.3, 0.7, 0.4, 1.0, 40, 1, 15, ci.BE, ci.DIRECT),
         ci.Problem(0.45, 0.6, 0.7, 0.5, 33, 2, 7, ci.BE, ci.DIRECT),
         ci.Problem(0.4, 0.6, 0.4, 1.0, 50, 1, 21, ci.BDF2, ci.DIRECT),
         ci.Problem(0.25, 0.8, 0.0, 1.0, 29, 2, 5, ci.BDF2, ci.DIRECT),
         ci.Problem(0.5, 0.5, 0.45, 1.0, 3, 1, 4, ci.BDF2, ci.DIRECT),
         ci.Problem(0.6, 0.3, 0.3, 1.0, 1, 1, 3, ci.BE, ci.DIRECT)]


@pytest.mark.parametrize("prec", [0, 4], ids=["f64", "df64"])
@pytest.mark.parametrize("p", CASES)
def test_gradient_against_oracle_adjoint(fc, p, prec):
    """FP64 and double-float (CQ_DF64: double-float histories, FP64 steps) gradients."""
    G0 = ci.g0_uniform(p.M, p.dim, 31)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 32)
    J, dG0, da = _grad(fc, p, G0, Gt, prec)
    Jr, dG0r, dar = AD.gradient(p, G0, Gt)
    assert abs(J - Jr) <= 1e-12 * abs(Jr)
    assert np.all(np.abs(da - dar) <= 1e-9 * np.abs(dar) + 1e-14 * abs(Jr))
    assert np.max(np.abs(dG0 - dG0r)) <= 1e-10 * np.max(np.abs(dG0r))


@pytest.mark.parametrize("prec", [0, 4], ids=["f64", "df64"])
@pytest.mark.parametrize("scheme", [ci.BE, ci.BDF2])
def test_gradient_against_finite_differences(fc, scheme, prec):
    """Misfit against a target made by the same scheme with perturbed orders,
    alpha + (0.05, -0.05), on a 2D grid; the finite differences of the FP64 forward solve."""
    p = ci.Problem(0.4, 0.6, 0.4, 1.0, 256, 2, 31, scheme, ci.DIRECT)
    G0 = ci.g0_checkerboard_uniform(p.M, ci.SEED_BASE + 9)
    cp_t = _cp(fc, p.replace(alpha1=0.45, alpha2=0.55))
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gt = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp_t, g0, gt, None), "cuda")
    fc.fp2s_solve(cp_t, g0, gt, ws)
    Gt = gt.cpu().numpy()
    J, dG0, da = _grad(fc, p, G0, Gt, prec)
    eps = 1e-5
    for s, f in ((0, "alpha1"), (1, "alpha2")):
        v = getattr(p, f)
        fd = (_J_gpu(fc, p.replace(**{f: v + eps}), G0, Gt) - _J_gpu(fc, p.replace(**{f: v - eps}), G0, Gt)) / (2 * eps)
        print("dJ/d%s adjoint %.12e fd %.12e rel %.2e" % (f, da[s], fd, abs(da[s] - fd) / abs(fd)))
        assert abs(da[s] - fd) <= 1e-6 * abs(fd)
    rng = np.random.default_rng(4)
    for _ in range(3):
        s, k = int(rng.integers(2)), int(rng.integers(G0.shape[1]))
        E = np.zeros_like(G0)
        E[s, k] = 1e-4
        fd = (_J_gpu(fc, p, G0 + E, Gt) - _J_gpu(fc, p, G0 - E, Gt)) / 2e-4
        assert abs(dG0[s, k] - fd) <= 1e-6 * np.max(np.abs(dG0))


@pytest.mark.parametrize("prec", [0, 4], ids=["f64", "df64"])
def test_gradient_in_mode_slices(fc, prec):
    """A workspace too small for all modes: the forward and adjoint sweeps run over slices of
    modes (independent in the sine basis); same per-mode arithmetic, so dJ/dG0 agrees to
    rounding and J, dJ/dalpha differ only in the order of their sums."""
    import ctypes as C
    p = ci.Problem(0.35, 0.6, 0.4, 1.0, 300, 2, 31, ci.BDF2, ci.DIRECT)
    G0 = ci.g0_uniform(p.M, p.dim, 41)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 42)
    J, dG0, da = _grad(fc, p, G0, Gt, prec)
    cp = _cp(fc, p, prec)
    full = fc.fp2s_gradient(cp, None, None, None, None)
    Jc, dac = C.c_double(0.0), (C.c_double * 2)()
    sz = C.c_size_t(full // 5)
    assert fc._lib.fp2s_gradient(C.byref(cp), None, None, C.byref(Jc), None, dac, None, C.byref(sz), None) == fc.CQ_OK
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gt = torch.tensor(Gt, dtype=torch.float64, device="cuda")
    dg = torch.empty_like(g0)
    Js, das = fc.fp2s_gradient(cp, g0, gt, dg, ws)
    assert abs(Js - J) <= 1e-13 * abs(J)
    assert np.all(np.abs(np.array(das) - da) <= 1e-12 * np.abs(da))
    assert np.max(np.abs(dg.cpu().numpy() - dG0)) <= 1e-13 * np.max(np.abs(dG0))
