"""GPU gradient of the fast form (fp2s_gradient / fp2s_vjp with CQ_FAST: the discrete adjoint
of the fast scheme, with backward geometric recurrences per quadrature node, in FP64 and with the
backward sweep in double-float, CQ_DF64) against the oracle's fast-scheme gradient and against
central finite differences of the GPU fast forward solve (``-m gpu``).

Tolerances: J to 1e-12 relative (the fast forward solve, parity-tested at 1e-12); dJ/dG0 to
1e-10 of its largest entry (sums over modes and steps whose rounding differs between the
sides); dJ/dalpha to 1e-8 relative: both sides take the beta-derivative of the quadrature
tables by extrapolated central differences of their own constructions (the GPU of the nodes
and coefficients, the oracle of the whole weight sequence), each accurate to ~1e-10. Central
differences of the forward solve (step 1e-5) are held to 1e-6 relative.
"""
import ctypes as C

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
    return fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, ci.FAST, p.np1, p.np2, p.ns,
                      prec=prec)


def _grad(fc, p, G0, Gt, cap=None, prec=0):
    cp = _cp(fc, p, prec)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gt = torch.tensor(Gt, dtype=torch.float64, device="cuda")
    dg = torch.empty_like(g0)
    if cap is None:
        ws = fc.workspace(fc.fp2s_gradient(cp, g0, gt, dg, None), "cuda")
    else:
        Jc, dac = C.c_double(0.0), (C.c_double * 2)()
        sz = C.c_size_t(cap)
        assert fc._lib.fp2s_gradient(C.byref(cp), None, None, C.byref(Jc), None, dac, None, C.byref(sz),
                                     None) == fc.CQ_OK
        ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    J, da = fc.fp2s_gradient(cp, g0, gt, dg, ws)
    return J, dg.cpu().numpy(), np.array(da)


def _J_gpu(fc, p, G0, Gt):
    cp = _cp(fc, p)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), "cuda")
    fc.fp2s_solve(cp, g0, gN, ws)
    h = 1.0 / (p.M + 1)
    return 0.5 * h ** p.dim * float(np.sum((gN.cpu().numpy() - Gt) ** 2))


CASES = [ci.Problem(0.3, 0.7, 0.4, 1.0, 60, 1, 15, ci.BE, ci.FAST, 16, 0, 2),
         ci.Problem(0.45, 0.6, 0.7, 0.5, 45, 2, 7, ci.BE, ci.FAST, 12, 0, 2),
         ci.Problem(0.4, 0.6, 0.4, 1.0, 70, 1, 21, ci.BDF2, ci.FAST, 6, 18, 9),
         ci.Problem(0.25, 0.8, 0.0, 1.0, 40, 2, 5, ci.BDF2, ci.FAST, 4, 12, 6),
         ci.Problem(0.5, 0.35, 0.45, 1.0, 4, 1, 4, ci.BDF2, ci.FAST, 3, 5, 7),
         ci.Problem(0.6, 0.3, 0.3, 1.0, 1, 1, 3, ci.BE, ci.FAST, 8, 0, 2),
         ci.Problem(0.35, 0.55, 0.6, 1.0, 50, 2, 9, ci.BDF2, ci.FAST, 7, 25, 17),
         ci.Problem(0.3, 0.6, 0.4, 1.0, 80, 1, 20, ci.BE, ci.FAST, 200, 0, 2),
         ci.Problem(0.45, 0.5, 0.35, 1.0, 90, 2, 6, ci.BDF2, ci.FAST, 40, 150, 32)]


@pytest.mark.parametrize("prec", [0, 4], ids=["f64", "df64"])
@pytest.mark.parametrize("p", CASES, ids=["be1d", "be2d", "bdf2_1d", "bdf2_2d_m0", "n_below_L", "one_step",
                                          "bdf2_ns17_idle_lanes", "be_np200", "bdf2_np190_ns32"])
def test_fast_gradient_against_oracle(fc, p, prec):
    if prec == 4 and p.np1 + p.np2 > 128:
        pytest.skip("the double-float fast form takes np1 + np2 <= 128")
    G0 = ci.g0_uniform(p.M, p.dim, 51)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 52)
    J, dG0, da = _grad(fc, p, G0, Gt, prec=prec)
    Jr, dG0r, dar = AD.gradient_fast(p, G0, Gt)
    print("J %.3e vs %.3e; dJ/dalpha rel %.2e %.2e; dJ/dG0 %.2e" % (
        J, Jr, *(np.abs(da - dar) / np.abs(dar)), np.max(np.abs(dG0 - dG0r)) / np.max(np.abs(dG0r))))
    assert abs(J - Jr) <= 1e-12 * abs(Jr)
    assert np.all(np.abs(da - dar) <= 1e-8 * np.abs(dar) + 1e-14 * abs(Jr))
    assert np.max(np.abs(dG0 - dG0r)) <= 1e-10 * np.max(np.abs(dG0r))


@pytest.mark.parametrize("prec", [0, 4], ids=["f64", "df64"])
@pytest.mark.parametrize("scheme", [ci.BE, ci.BDF2])
def test_fast_gradient_against_finite_differences(fc, scheme, prec):
    """Misfit against a target made by the same fast scheme with alpha + (0.05, -0.05) on a
    2D grid; central differences of the GPU fast forward solve (tables rebuilt at alpha +- eps)."""
    np1, np2, ns = (32, 0, 2) if scheme == ci.BE else (16, 48, 17)
    p = ci.Problem(0.4, 0.6, 0.4, 1.0, 512, 2, 31, scheme, ci.FAST, np1, np2, ns)
    G0 = ci.g0_checkerboard_uniform(p.M, ci.SEED_BASE + 9)
    cp_t = _cp(fc, p.replace(alpha1=0.45, alpha2=0.55))
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gt = torch.empty_like(g0)
    fc.fp2s_solve(cp_t, g0, gt, fc.workspace(fc.fp2s_solve(cp_t, g0, gt, None), "cuda"))
    Gt = gt.cpu().numpy()
    J, dG0, da = _grad(fc, p, G0, Gt, prec=prec)
    eps = 1e-5
    for s, f in ((0, "alpha1"), (1, "alpha2")):
        v = getattr(p, f)
        fd = (_J_gpu(fc, p.replace(**{f: v + eps}), G0, Gt) - _J_gpu(fc, p.replace(**{f: v - eps}), G0, Gt)) / (2 * eps)
        print("fast dJ/d%s adjoint %.12e fd %.12e rel %.2e" % (f, da[s], fd, abs(da[s] - fd) / abs(fd)))
        assert abs(da[s] - fd) <= 1e-6 * abs(fd)
    rng = np.random.default_rng(6)
    for _ in range(3):
        s, k = int(rng.integers(2)), int(rng.integers(G0.shape[1]))
        E = np.zeros_like(G0)
        E[s, k] = 1e-4
        fd = (_J_gpu(fc, p, G0 + E, Gt) - _J_gpu(fc, p, G0 - E, Gt)) / 2e-4
        assert abs(dG0[s, k] - fd) <= 1e-6 * np.max(np.abs(dG0))


def test_fast_vjp_dot_product(fc):
    """<vjp(Y), V> = <G^N(V), Y>: the fast forward solve is linear in G^0 and the vjp is its
    transpose, to rounding."""
    p = ci.Problem(0.3, 0.7, 0.45, 1.0, 400, 2, 15, ci.BDF2, ci.FAST, 8, 24, 9)
    rng = np.random.default_rng(12)
    V = rng.standard_normal((2, p.M ** 2))
    Y = rng.standard_normal((2, p.M ** 2))
    cp = _cp(fc, p)
    v = torch.tensor(V, dtype=torch.float64, device="cuda")
    y = torch.tensor(Y, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(v)
    fc.fp2s_solve(cp, v, gN, fc.workspace(fc.fp2s_solve(cp, v, gN, None), "cuda"))
    dg = torch.empty_like(v)
    fc.fp2s_vjp(cp, v, y, dg, fc.workspace(fc.fp2s_vjp(cp, v, y, dg, None), "cuda"))
    lhs = float(torch.sum(dg * v))
    rhs = float(torch.sum(gN * y))
    print("fast dot-product test: <vjp(Y),V> %.15e <G^N(V),Y> %.15e" % (lhs, rhs))
    assert abs(lhs - rhs) <= 1e-12 * float(torch.linalg.norm(dg) * torch.linalg.norm(v))


@pytest.mark.parametrize("prec", [0, 4], ids=["f64", "df64"])
def test_fast_gradient_in_mode_slices(fc, prec):
    """A workspace cap below the unsliced size: forward and adjoint sweeps over slices of modes
    give the same dJ/dG0 per mode and J, dJ/dalpha up to the order of their sums."""
    p = ci.Problem(0.35, 0.6, 0.4, 1.0, 300, 2, 31, ci.BDF2, ci.FAST, 8, 24, 9)
    G0 = ci.g0_uniform(p.M, p.dim, 53)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 54)
    J, dG0, da = _grad(fc, p, G0, Gt, prec=prec)
    full = fc.fp2s_gradient(_cp(fc, p, prec), None, None, None, None)
    Js, dGs, das = _grad(fc, p, G0, Gt, cap=full // 5, prec=prec)
    assert abs(Js - J) <= 1e-13 * abs(J)
    assert np.all(np.abs(das - da) <= 1e-12 * np.abs(da))
    assert np.max(np.abs(dGs - dG0)) <= 1e-13 * np.max(np.abs(dG0))


def test_fast_gradient_double_float_against_fp64(fc):
    """The double-float backward sweep against the FP64 one on the 2D 63x63 grid (BDF2, 16 + 64
    points, Ns = 17, N = 1024): the same forward levels, so the two differ by the double-float
    rounding of the recurrences (~2^-48 per operation), far inside 1e-9."""
    p = ci.Problem(0.4, 0.6, 0.4, 1.0, 1024, 2, 63, ci.BDF2, ci.FAST, 16, 64, 17)
    G0 = ci.g0_checkerboard_uniform(p.M, ci.SEED_BASE + 11)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 55)
    J, dG0, da = _grad(fc, p, G0, Gt)
    Jd, dGd, dad = _grad(fc, p, G0, Gt, prec=4)
    print("double-float vs FP64 fast gradient: J %.2e, dJ/dalpha %.2e %.2e, dJ/dG0 %.2e" % (
        abs(Jd - J) / abs(J), *(np.abs(dad - da) / np.abs(da)), np.max(np.abs(dGd - dG0)) / np.max(np.abs(dG0))))
    assert abs(Jd - J) <= 1e-13 * abs(J)
    assert np.all(np.abs(dad - da) <= 1e-9 * np.abs(da))
    assert np.max(np.abs(dGd - dG0)) <= 1e-10 * np.max(np.abs(dG0))
