"""GPU parity of the double-float solves (precision form CQ_DF64, fast and direct, ``-m gpu``).

The fast history's node states, tables and sums are pairs of FP32 numbers (about 48
significant bits) on the FP32 pipe, the 2x2 step is FP64. It is held to the FP64 bar
of the fast form: against the oracle's FP64 fast scheme (same tables), relative L2
error <= 1e-12 per state and max element error <= 1e-11 * max|ref|, and against the
GPU's FP64 fast solve the same. The cases cover both schemes, 1D/2D/3D grids, every
compile-time node bound (16 .. 128 points per state, ragged counts; above 80 the
fastest-decaying slots live in shared memory), the few-mode sizes,
and the power-of-two rescaling that keeps every mode inside the FP32 exponent range
(fields near 2^+-900 and a growing mode).
"""
import numpy as np
import pytest

import cq_inputs as ci
from oracle import scheme as OS
from oracle import spatial as OSP

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
    return fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                      prec=prec)


def _solve(fc, p, G0, prec):
    cp = _cp(fc, p, prec)
    g0 = torch.tensor(np.ascontiguousarray(G0), dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), "cuda")
    st = fc.fp2s_solve(cp, g0, gN, ws, check=False)
    torch.cuda.synchronize()
    return gN.cpu().numpy(), st


def _assert_close(got, ref, tag):
    errs = []
    for s in range(2):
        sc = np.max(np.abs(ref[s]))
        errs.append(float(np.linalg.norm((got[s] - ref[s]) / sc) / np.linalg.norm(ref[s] / sc)))
    print("%s: rel L2 per state %.3e %.3e" % (tag, *errs))
    assert max(errs) <= 1e-12
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


CASES = [
    ("be1d_np64", ci.Problem(0.3, 0.7, 0.4, 1.0, 1024, 1, 63, ci.BE, ci.FAST, 64, 0, 2)),
    ("bdf2_1d_np80", ci.Problem(0.4, 0.6, 0.3, 1.0, 700, 1, 45, ci.BDF2, ci.FAST, 16, 64, 17)),
    ("be2d_np40", ci.Problem(0.25, 0.55, 0.7, 0.5, 333, 2, 21, ci.BE, ci.FAST, 40, 0, 2)),
    ("bdf2_2d_np32", ci.Problem(0.2, 0.8, 0.45, 1.0, 257, 2, 19, ci.BDF2, ci.FAST, 9, 23, 7)),
    ("bdf2_2d_np16_many", ci.Problem(0.35, 0.65, 0.2, 1.0, 300, 2, 127, ci.BDF2, ci.FAST, 6, 10, 5)),
    ("be2d_np80_many", ci.Problem(0.2, 0.8, 0.45, 1.0, 500, 2, 131, ci.BE, ci.FAST, 80, 0, 2)),
    ("bdf2_3d_np42", ci.Problem(0.3, 0.6, 0.65, 1.0, 150, 3, 11, ci.BDF2, ci.FAST, 12, 30, 9)),
    ("be3d_ragged", ci.Problem(0.6, 0.45, 0.3, 0.5, 77, 3, 13, ci.BE, ci.FAST, 37, 0, 2)),
    ("tiny", ci.Problem(0.5, 0.5, 0.6, 1.0, 3, 1, 1, ci.BDF2, ci.FAST, 2, 2, 3)),
    ("one_step_bdf2", ci.Problem(0.5, 0.5, 0.6, 1.0, 1, 2, 3, ci.BDF2, ci.FAST, 4, 4, 3)),
    ("two_steps_be", ci.Problem(0.3, 0.7, 0.4, 1.0, 2, 1, 5, ci.BE, ci.FAST, 8, 0, 2)),
    ("bdf2_ns32", ci.Problem(0.45, 0.55, 0.35, 1.0, 400, 2, 33, ci.BDF2, ci.FAST, 20, 40, 32)),
    ("m0_coupled", ci.Problem(0.3, 0.8, 0.0, 1.0, 400, 2, 47, ci.BDF2, ci.FAST, 16, 48, 15)),
    # more than 80 points: the fastest-decaying slots in shared memory
    ("be2d_np128", ci.Problem(0.2, 0.8, 0.45, 1.0, 700, 2, 63, ci.BE, ci.FAST, 128, 0, 2)),
    ("bdf2_2d_np112", ci.Problem(0.35, 0.55, 0.6, 1.0, 500, 2, 63, ci.BDF2, ci.FAST, 16, 96, 17)),
    ("bdf2_1d_np90_ns20", ci.Problem(0.6, 0.25, 0.35, 1.0, 600, 1, 255, ci.BDF2, ci.FAST, 30, 60, 20)),
]


@pytest.mark.parametrize("name,p", CASES, ids=[c[0] for c in CASES])
def test_df64_solve_matches_oracle_and_fp64(fc, name, p):
    G0 = ci.g0_uniform(p.M, p.dim, 71)
    got, st = _solve(fc, p, G0, fc.CQ_DF64)
    assert st == fc.CQ_OK
    _assert_close(got, OS.solve(p, G0), name + " vs oracle")
    f64, st64 = _solve(fc, p, G0, fc.CQ_F64)
    assert st64 == fc.CQ_OK
    _assert_close(got, f64, name + " vs FP64 kernel")


@pytest.mark.parametrize("e", [900, -900])
def test_df64_extreme_scales(fc, e):
    """Fields of size 2^+-900 lie far outside the FP32 range: the per-mode power-of-two
    scaling brings them in, and the result is the scaled result of the unscaled field."""
    p = ci.Problem(0.4, 0.6, 0.3, 1.0, 600, 2, 63, ci.BDF2, ci.FAST, 16, 64, 17)
    G0 = ci.g0_uniform(p.M, p.dim, 72)
    got, st = _solve(fc, p, G0 * 2.0 ** e, fc.CQ_DF64)
    assert st == fc.CQ_OK
    ref = OS.solve(p, G0)
    _assert_close(got * 2.0 ** -e, ref, "G0 x 2^%d" % e)


def test_df64_growing_mode_rescaled(fc):
    """m = 0.49 on a 1D grid (T = 0.4): the lowest mode grows like e^(2448 t), past 2^1400 over
    the run, so the solve rescales it by 2^40 dozens of times. In the sine basis (G0 x 2^-1000,
    so that the oracle's FP64 stays finite) the decaying modes match the oracle at the FP64
    bar, and each growing mode within 4 x its one-ulp conditioning (the largest change of the
    oracle's g^N when lambda_k, a or T moves by one ulp), as in the FP64 sine-basis test."""
    p = ci.Problem(0.4, 0.6, 0.49, 0.4, 2048, 1, 255, ci.BDF2, ci.FAST, 16, 64, 17)
    lam = OSP.mode_eigenvalues(p.M, p.dim)
    rates = np.array([ci.growth_rate(p.alpha1, p.alpha2, p.m, l_) for l_ in lam[:8]])
    assert rates[0] * p.T > 1200 * np.log(2.0)          # grows past 2^1200: many rescales
    # only the growing modes are scaled down (modes are independent), so that the decaying
    # ones stay far from the FP64 subnormal range in the oracle
    g0m = OSP.to_modal(ci.g0_uniform(p.M, p.dim, 73), p.M, p.dim)
    g0m[:, :8] *= np.where(rates > 0, 2.0 ** -1000, 1.0)[None, :]
    cp = _cp(fc, p, fc.CQ_DF64)
    g0 = torch.tensor(g0m, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve_modes(cp, 0, p.M, g0, gN, None), "cuda")
    assert fc.fp2s_solve_modes(cp, 0, p.M, g0, gN, ws, check=False) == fc.CQ_OK
    got = gN.cpu().numpy()
    ref = OS.solve_modal(p, lam, g0m)[p.N]
    assert np.all(np.isfinite(ref))
    one_ulp = 2.0 ** -52
    for k in np.where(rates > 0)[0]:
        lam_k, g0_k = lam[[k]], g0m[:, [k]]
        moved = [OS.solve_modal(p, lam_k * (1 + one_ulp), g0_k)[p.N],
                 OS.solve_modal(p, lam_k, g0_k, a=OS.coupling(p.m) * (1 + one_ulp))[p.N],
                 OS.solve_modal(p.replace(T=p.T * (1 + one_ulp)), lam_k, g0_k)[p.N]]
        kappa = max(float(np.max(np.abs(m_ - ref[:, [k]])) / np.max(np.abs(ref[:, k]))) for m_ in moved)
        err = float(np.max(np.abs(got[:, k] - ref[:, k])) / np.max(np.abs(ref[:, k])))
        print("growing mode %d (rate %.1f): rel error %.3e, one-ulp conditioning %.3e" % (k, rates[k], err, kappa))
        assert err <= 4.0 * kappa
    calm = np.arange(8, p.M)
    _assert_close(got[:, calm], ref[:, calm], "decaying modes")


DIRECT_CASES = [
    ("be1d_m63", ci.Problem(0.3, 0.7, 0.4, 1.0, 1024, 1, 63, ci.BE, ci.DIRECT)),
    ("bdf2_1d", ci.Problem(0.4, 0.6, 0.3, 1.0, 700, 1, 45, ci.BDF2, ci.DIRECT)),
    ("bdf2_2d_m0", ci.Problem(0.2, 0.8, 0.0, 1.0, 257, 2, 19, ci.BDF2, ci.DIRECT)),
    ("be2d_ragged_N", ci.Problem(0.25, 0.55, 0.7, 0.5, 333, 2, 41, ci.BE, ci.DIRECT)),
    ("be3d", ci.Problem(0.35, 0.7, 0.4, 1.0, 120, 3, 9, ci.BE, ci.DIRECT)),
    ("tiny", ci.Problem(0.5, 0.5, 0.6, 1.0, 3, 1, 1, ci.BDF2, ci.DIRECT)),
    ("one_step", ci.Problem(0.5, 0.5, 0.6, 1.0, 1, 2, 3, ci.BE, ci.DIRECT)),
    ("two_steps_bdf2", ci.Problem(0.4, 0.6, 0.3, 1.0, 2, 1, 7, ci.BDF2, ci.DIRECT)),
    ("one_step_bdf2", ci.Problem(0.4, 0.6, 0.3, 1.0, 1, 2, 5, ci.BDF2, ci.DIRECT)),
    ("bdf2_2d_many", ci.Problem(0.45, 0.65, 0.35, 1.0, 600, 2, 127, ci.BDF2, ci.DIRECT)),
]


@pytest.mark.parametrize("name,p", DIRECT_CASES, ids=[c[0] for c in DIRECT_CASES])
def test_df64_direct_matches_oracle_and_fp64(fc, name, p):
    """The direct scheme with double-float weights, levels and history sums (FP64 step)."""
    G0 = ci.g0_uniform(p.M, p.dim, 81)
    got, st = _solve(fc, p, G0, fc.CQ_DF64)
    assert st == fc.CQ_OK
    _assert_close(got, OS.solve(p, G0), name + " direct vs oracle")
    f64, st64 = _solve(fc, p, G0, fc.CQ_F64)
    assert st64 == fc.CQ_OK
    _assert_close(got, f64, name + " direct vs FP64 kernel")


def test_df64_direct_full_size_decaying_modes(fc):
    """The 2D 255x255 BDF2 workload (N = 4096, m = 0.49) in the direct double-float form over
    the modes past the second row of the spectrum (the three growing modes, whose growth of
    up to e^1096 leaves the FP32 exponent range, lie before it), in the sine basis against
    the oracle's FP64 direct scheme on seeded sampled modes: relative L2 per state <= 1e-12."""
    p, G0 = ci.workload("bdf2_2d_m255")
    p = p.replace(form=ci.DIRECT)
    nm = p.M ** p.dim
    lo = p.M + 1
    g0m = OSP.to_modal(G0, p.M, p.dim)
    cp = _cp(fc, p, fc.CQ_DF64)
    g0 = torch.tensor(np.ascontiguousarray(g0m[:, lo:]), dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve_modes(cp, lo, nm, g0, gN, None), "cuda")
    assert fc.fp2s_solve_modes(cp, lo, nm, g0, gN, ws, check=False) == fc.CQ_OK
    got = gN.cpu().numpy()
    sample = np.unique(np.concatenate([[0, 1, 2], ci.sample_indices(nm - lo, 40, ci.SEED_BASE + 14)]))
    lam = OSP.mode_eigenvalues(p.M, p.dim)[lo + sample]
    ref = OS.solve_modal(p, lam, g0m[:, lo + sample])[p.N]
    _assert_close(got[:, sample], ref, "direct df64 full size")
