"""Gradient through the mixed-precision direct solve (fp2s_gradient / fp2s_vjp with
prec = CQ_BF16X3 or CQ_TF32X3) against the FP64 oracle adjoint and the FP64 GPU
gradient (``-m gpu``).

The forward solve, the weight-derivative history sum_{k<=n} d'_{n-k} x^k and the
reversed-time adjoint all run on FP32 levels with tensor-core histories, so each carries
the error level of the mixed forward solve (relative ~1e-6 .. 3e-6, see
test_gpu_mixed.py). The gradients are sums of products of the two sweeps and inherit
that level. Bars: J and dJ/dG0 (relative L2) within 5e-5 (measured <= 4.3e-6), dJ/dalpha
within 5e-4 relative (sums over all modes and steps, with partial cancellation between
them; measured <= 1.3e-4 on the one-step cases, where dJ/dalpha is smallest).
The measured values are printed.
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


def _cp(fc, p, prec):
    return fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, ci.DIRECT, prec=prec)


def _grad(fc, p, G0, Gt, prec):
    cp = _cp(fc, p, prec)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gt = torch.tensor(Gt, dtype=torch.float64, device="cuda")
    dg = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_gradient(cp, g0, gt, dg, None), "cuda")
    J, da = fc.fp2s_gradient(cp, g0, gt, dg, ws)
    return J, dg.cpu().numpy(), np.array(da)


def _errs(J, dG0, da, Jr, dG0r, dar):
    return (abs(J - Jr) / abs(Jr), float(np.linalg.norm(dG0 - dG0r) / np.linalg.norm(dG0r)),
            np.abs(da - dar) / np.abs(dar))


CASES = [
    ("be_1d_3blocks", ci.Problem(0.3, 0.7, 0.4, 1.0, 300, 1, 31, ci.BE, ci.DIRECT)),
    ("bdf2_1d_3blocks", ci.Problem(0.4, 0.6, 0.3, 1.0, 260, 1, 31, ci.BDF2, ci.DIRECT)),
    ("bdf2_2d", ci.Problem(0.35, 0.65, 0.4, 1.0, 200, 2, 15, ci.BDF2, ci.DIRECT)),
    ("be_2d_one_block", ci.Problem(0.45, 0.6, 0.7, 0.5, 100, 2, 9, ci.BE, ci.DIRECT)),
    ("bdf2_1d_block_plus_one", ci.Problem(0.25, 0.8, 0.45, 1.0, 129, 1, 17, ci.BDF2, ci.DIRECT)),
    ("bdf2_1d_two_pairs", ci.Problem(0.3, 0.5, 0.35, 1.0, 513, 1, 9, ci.BDF2, ci.DIRECT)),
    ("bdf2_1d_m0_N3", ci.Problem(0.5, 0.5, 0.0, 1.0, 3, 1, 4, ci.BDF2, ci.DIRECT)),
    ("bdf2_1d_N2", ci.Problem(0.3, 0.7, 0.4, 1.0, 2, 1, 5, ci.BDF2, ci.DIRECT)),
    ("bdf2_1d_N1", ci.Problem(0.3, 0.7, 0.4, 1.0, 1, 1, 5, ci.BDF2, ci.DIRECT)),
    ("be_1d_N1", ci.Problem(0.6, 0.3, 0.3, 0.5, 1, 1, 3, ci.BE, ci.DIRECT)),
    ("be_1d_strong_coupling", ci.Problem(0.4, 0.6, 0.48, 1.0, 150, 1, 15, ci.BE, ci.DIRECT)),
]


@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_mixed_gradient_against_oracle_adjoint(fc, name, p):
    G0 = ci.g0_uniform(p.M, p.dim, 31)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 32)
    Jr, dG0r, dar = AD.gradient(p, G0, Gt)
    for prec in (fc.CQ_BF16X3, fc.CQ_TF32X3):
        eJ, eG, ea = _errs(*_grad(fc, p, G0, Gt, prec), Jr, dG0r, dar)
        print("mixed gradient %s prec %d: J %.2e dG0 %.2e dalpha %.2e %.2e" % (name, prec, eJ, eG, ea[0], ea[1]))
        assert eJ <= 5e-5 and eG <= 5e-5
        assert np.all(ea <= 5e-4)


def test_mixed_vjp_matches_mixed_gradient(fc):
    """fp2s_vjp with dL/dG^N = h^d (G^N - Gt), G^N from the mixed solve, equals fp2s_gradient."""
    p = ci.Problem(0.35, 0.65, 0.4, 1.0, 300, 2, 15, ci.BDF2, ci.DIRECT)
    G0 = ci.g0_uniform(p.M, p.dim, 5)
    Gt = 0.3 * ci.g0_uniform(p.M, p.dim, 6)
    cp = _cp(fc, p, fc.CQ_BF16X3)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), "cuda")
    fc.fp2s_solve(cp, g0, gN, ws)
    h = 1.0 / (p.M + 1)
    dGN = h ** p.dim * (gN - torch.tensor(Gt, dtype=torch.float64, device="cuda"))
    dg = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_vjp(cp, g0, dGN, dg, None), "cuda")
    da = np.array(fc.fp2s_vjp(cp, g0, dGN, dg, ws))
    _, dG0, da_g = _grad(fc, p, G0, Gt, fc.CQ_BF16X3)
    assert np.linalg.norm(dg.cpu().numpy() - dG0) <= 1e-6 * np.linalg.norm(dG0)
    assert np.all(np.abs(da - da_g) <= 1e-6 * np.abs(da_g))


def test_mixed_vjp_dot_product(fc):
    """<vjp(Y), V> = <G^N(V), Y> (G^N is linear in G^0): both sides from the mixed forms."""
    p = ci.Problem(0.3, 0.7, 0.45, 1.0, 400, 1, 63, ci.BE, ci.DIRECT)
    rng = np.random.default_rng(11)
    V = rng.standard_normal((2, p.M))
    Y = rng.standard_normal((2, p.M))
    cp = _cp(fc, p, fc.CQ_BF16X3)
    v = torch.tensor(V, dtype=torch.float64, device="cuda")
    y = torch.tensor(Y, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(v)
    ws = fc.workspace(fc.fp2s_solve(cp, v, gN, None), "cuda")
    fc.fp2s_solve(cp, v, gN, ws)
    dg = torch.empty_like(v)
    ws = fc.workspace(fc.fp2s_vjp(cp, v, y, dg, None), "cuda")
    fc.fp2s_vjp(cp, v, y, dg, ws)
    lhs = float(torch.sum(dg * v))
    rhs = float(torch.sum(gN * y))
    print("mixed dot-product test: <vjp(Y),V> %.12e <G^N(V),Y> %.12e" % (lhs, rhs))
    assert abs(lhs - rhs) <= 1e-4 * float(torch.linalg.norm(dg) * torch.linalg.norm(v))


def test_mixed_gradient_full_size(fc):
    """The 2D 255x255, N = 4096 gradient workload (BDF2, alpha = (0.4, 0.6), m = 0.4,
    target from alpha + (0.05, -0.05)): mixed against the FP64 GPU gradient, which the
    oracle adjoint and central differences pin on smaller problems. The forward and the
    adjoint sweep each carry the FP32 level of the mixed forward solve: J and dJ/dG0 are held
    to 1e-4 (measured 6e-6 .. 2.4e-5) and dJ/dalpha to 1e-4 (measured 6e-6 .. 1.5e-5)."""
    p, G0, Gt = _grad_workload(fc)
    J64, dG64, da64 = _grad(fc, p, G0, Gt, fc.CQ_F64)
    for prec in (fc.CQ_BF16X3, fc.CQ_TF32X3):
        eJ, eG, ea = _errs(*_grad(fc, p, G0, Gt, prec), J64, dG64, da64)
        print("mixed gradient full size prec %d: J %.2e dG0 %.2e dalpha %.2e %.2e" % (prec, eJ, eG, ea[0], ea[1]))
        assert eJ <= 1e-4 and eG <= 1e-4
        assert np.all(ea <= 1e-4)


def _grad_workload(fc):
    p, G0 = ci.workload("grad_2d_m255")
    cp_t = _cp(fc, p.replace(alpha1=p.alpha1 + 0.05, alpha2=p.alpha2 - 0.05), fc.CQ_F64)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gt = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp_t, g0, gt, None), "cuda")
    fc.fp2s_solve(cp_t, g0, gt, ws)
    return p, G0, gt.cpu().numpy()


@pytest.mark.parametrize("prec", [2, 3])
def test_mixed_gradient_in_mode_slices(fc, prec):
    """A workspace too small for all modes: the mixed-precision forward and adjoint sweeps run
    over slices of modes (independent in the sine basis; multiples of 64 modes, the last one
    ragged). Each mode takes the same arithmetic as in the unsliced run, so dJ/dG0 agrees to
    rounding of its transform, and J, dJ/dalpha differ only in the order of their FP64 sums."""
    import ctypes as C
    p = ci.Problem(0.35, 0.6, 0.4, 1.0, 300, 2, 31, ci.BDF2, ci.DIRECT)
    G0 = ci.g0_uniform(p.M, p.dim, 41)
    Gt = 0.5 * ci.g0_uniform(p.M, p.dim, 42)
    J, dG0, da = _grad(fc, p, G0, Gt, prec)
    cp = _cp(fc, p, prec)
    full = fc.fp2s_gradient(cp, None, None, None, None)
    Jc, dac = C.c_double(0.0), (C.c_double * 2)()
    sz = C.c_size_t(full // 4)
    assert fc._lib.fp2s_gradient(C.byref(cp), None, None, C.byref(Jc), None, dac, None, C.byref(sz), None) == fc.CQ_OK
    assert sz.value <= full // 4
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gt = torch.tensor(Gt, dtype=torch.float64, device="cuda")
    dg = torch.empty_like(g0)
    Js, das = fc.fp2s_gradient(cp, g0, gt, dg, ws)
    print("mixed gradient in slices (prec %d, %d of %d bytes): J %.2e dalpha %s" % (
        prec, sz.value, full, abs(Js - J) / abs(J), np.abs(np.array(das) - da) / np.abs(da)))
    assert abs(Js - J) <= 1e-12 * abs(J)
    assert np.all(np.abs(np.array(das) - da) <= 1e-12 * np.abs(da))
    assert np.max(np.abs(dg.cpu().numpy() - dG0)) <= 1e-13 * np.max(np.abs(dG0))
    # a cap below one slice of 64 modes is refused
    sz = C.c_size_t(4096)
    assert fc._lib.fp2s_gradient(C.byref(cp), None, None, C.byref(Jc), None, dac, None, C.byref(sz),
                                 None) == fc.CQ_ENOMEM
