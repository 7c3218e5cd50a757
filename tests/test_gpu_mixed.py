"""Mixed-precision direct solve (form = CQ_DIRECT, prec = CQ_BF16X3 / CQ_TF32X3) against
the FP64 oracle (``-m gpu``).

The history of Eq. 3.8 is split per time block of 128 steps: the part from earlier
blocks is a tensor-core contraction of split operands (BF16 hi + lo: <= 3 * 2^-16 per term;
TF32 hi + lo: <= 3 * 2^-22) accumulated in FP32 per chunk and summed across chunks with
round-to-nearest; the in-block part is an FP32 sum; the step (Eq. 4.1 / Eq. 4.7) is
x = A l + B e with double-float A and B (FP64 when |a| > 10). Error sources of a slowly
varying mode (u = 2^-24):
- a systematic relative error eps in the history weights breaks their vanishing sum and
  acts like a reaction term (a + lambda) eps tau^-beta: the FP32 rounding of d_1 ~ beta
  tau^-beta and d_2 is therefore carried as a remainder term in the step, and the
  tensor-core accumulator, which truncates toward zero at every MMA instruction, is read
  back per chunk (128 BF16 / 32 TF32 levels) with the small products issued first;
- random per-step roundings of the FP32 levels and sums add up like a random walk: ~1e-6
  at N = 8192; the BF16 split of the levels (2^-17 per level) adds ~3e-6.
Bars: relative L2 error per state at the final step <= 2e-5 (BF16x3) and 1e-5 (TF32x3),
measured <= 3.4e-6 and 2.2e-6 on these cases (printed).
"""
import numpy as np
import pytest

import cq_inputs as ci
from oracle import scheme as OS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_05128_gb300 as pkg
    pkg.build()
    return pkg.load()


def _solve(fc, p, G0, prec):
    cp = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                    prec=prec)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), "cuda")
    st = fc.fp2s_solve(cp, g0, gN, ws, check=False)
    torch.cuda.synchronize()
    return gN.cpu().numpy(), st


def _rel(got, ref):
    return [float(np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s])) for s in range(2)]


MIXED_CASES = [
    # name, problem (form DIRECT), G0 scale exponent
    ("be_1d_3blocks_ragged", ci.Problem(0.3, 0.7, 0.4, 1.0, 300, 1, 63, ci.BE, ci.DIRECT, 0, 0, 0), -200),
    ("bdf2_1d_8blocks", ci.Problem(0.4, 0.6, 0.3, 1.0, 1000, 1, 127, ci.BDF2, ci.DIRECT, 0, 0, 0), 0),
    ("bdf2_2d_ragged_tiles", ci.Problem(0.4, 0.6, 0.7, 1.0, 600, 2, 23, ci.BDF2, ci.DIRECT, 0, 0, 0), 300),
    ("be_2d_m0.45", ci.Problem(0.2, 0.8, 0.45, 1.0, 520, 2, 31, ci.BE, ci.DIRECT, 0, 0, 0), 0),
    ("bdf2_1d_m0.48_solve64", ci.Problem(0.5, 0.7, 0.48, 0.5, 400, 1, 31, ci.BDF2, ci.DIRECT, 0, 0, 0), 0),
    ("be_1d_one_block", ci.Problem(0.6, 0.3, 0.2, 1.0, 128, 1, 17, ci.BE, ci.DIRECT, 0, 0, 0), 0),
    ("bdf2_1d_block_plus_one", ci.Problem(0.6, 0.3, 0.6, 1.0, 129, 1, 17, ci.BDF2, ci.DIRECT, 0, 0, 0), 0),
    ("be_1d_N1", ci.Problem(0.3, 0.7, 0.4, 1.0, 1, 1, 9, ci.BE, ci.DIRECT, 0, 0, 0), 0),
    ("bdf2_3d", ci.Problem(0.35, 0.6, 0.4, 1.0, 300, 3, 15, ci.BDF2, ci.DIRECT, 0, 0, 0), 0),
    ("bdf2_1d_N2", ci.Problem(0.3, 0.7, 0.4, 1.0, 2, 1, 9, ci.BDF2, ci.DIRECT, 0, 0, 0), 0),
]


@pytest.mark.parametrize("name,p,sc", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_direct_mixed_against_fp64_oracle(fc, name, p, sc):
    G0 = ci.g0_uniform(p.M, p.dim, 23) * 2.0 ** sc
    got, st = _solve(fc, p, G0, fc.CQ_BF16X3)
    assert st == fc.CQ_OK
    ref = OS.solve(p, G0)
    errs = _rel(got, ref)
    print("mixed direct %s rel L2 errors %.3e %.3e" % (name, errs[0], errs[1]))
    assert max(errs) <= 2e-5


@pytest.mark.parametrize("name,p,sc", MIXED_CASES[:6], ids=[c[0] for c in MIXED_CASES[:6]])
def test_direct_mixed_tf32x3_against_fp64_oracle(fc, name, p, sc):
    """The TF32x3 contraction in the same block algorithm (its split error, 2^-22 per term,
    is below the FP32 level of the in-block sums and levels)."""
    G0 = ci.g0_uniform(p.M, p.dim, 23) * 2.0 ** sc
    got, st = _solve(fc, p, G0, fc.CQ_TF32X3)
    assert st == fc.CQ_OK
    errs = _rel(got, OS.solve(p, G0))
    print("mixed direct tf32x3 %s rel L2 errors %.3e %.3e" % (name, errs[0], errs[1]))
    assert max(errs) <= 1e-5


def test_direct_mixed_every_step_count(fc):
    """Final states of the mixed solve for every N in 1..40 and around the block and pair
    edges (each N is its own problem, tau = T / N), against the oracle."""
    worst = 0.0
    for N in list(range(1, 41)) + [127, 128, 129, 255, 256, 257, 383, 384, 385, 511, 512, 513, 640, 641]:
        p = ci.Problem(0.3, 0.6, 0.35, 1.0, N, 1, 15, ci.BDF2 if N % 2 else ci.BE, ci.DIRECT, 0, 0, 0)
        G0 = ci.g0_uniform(p.M, p.dim, 100 + N)
        got, st = _solve(fc, p, G0, fc.CQ_BF16X3)
        assert st == fc.CQ_OK, N
        errs = _rel(got, OS.solve(p, G0))
        worst = max(worst, max(errs))
        assert max(errs) <= 2e-5, N
    print("mixed direct, N in 1..40 and block edges: worst rel L2 error %.3e" % worst)


def test_direct_mixed_matches_fp64_gpu_solve(fc):
    """Same problem through the FP64 direct kernel and the mixed solve: agree to the bound."""
    p = ci.Problem(0.2, 0.8, 0.45, 1.0, 700, 2, 47, ci.BE, ci.DIRECT, 0, 0, 0)
    G0 = ci.g0_disc_gaussian(p.M, 5)
    g64, st64 = _solve(fc, p, G0, fc.CQ_F64)
    gmx, stmx = _solve(fc, p, G0, fc.CQ_BF16X3)
    assert st64 == fc.CQ_OK and stmx == fc.CQ_OK
    errs = _rel(gmx, g64)
    print("mixed vs FP64 GPU direct: %.3e %.3e" % tuple(errs))
    assert max(errs) <= 2e-5


def test_mixed_form_rejected_for_fast_and_stepper(fc):
    g0 = torch.zeros((2, 15), dtype=torch.float64, device="cuda")
    cf = fc.problem(0.3, 0.7, 0.3, 1.0, 64, 1, 15, fc.CQ_BE, fc.CQ_FAST, 16, 0, 2, prec=fc.CQ_BF16X3)
    with pytest.raises(fc.CQError) as e:
        fc.fp2s_solve(cf, g0, g0, None)
    assert e.value.status == fc.CQ_EUNSUPPORTED
    cd = fc.problem(0.3, 0.7, 0.3, 1.0, 64, 1, 15, fc.CQ_BE, fc.CQ_DIRECT, prec=fc.CQ_BF16X3)
    with pytest.raises(fc.CQError) as e:
        fc.fp2s_init(cd, g0, None)
    assert e.value.status == fc.CQ_EUNSUPPORTED


def test_timing_parts_of_the_mixed_solve(fc):
    """cq_timing_part(1) sums the contraction launches inside the timed region."""
    p = ci.Problem(0.2, 0.8, 0.45, 1.0, 900, 2, 31, ci.BE, ci.DIRECT, 0, 0, 0)
    G0 = ci.g0_uniform(p.M, p.dim, 3)
    fc.cq_timing_enable(True)
    try:
        _solve(fc, p, G0, fc.CQ_BF16X3)
        whole, part = fc.cq_timing_part(0), fc.cq_timing_part(1)
        assert whole == fc.cq_timing_last()
        assert 0.0 < part < whole
        _solve(fc, p, G0, fc.CQ_F64)
        assert fc.cq_timing_part(1) == 0.0
        with pytest.raises(fc.CQError):
            fc.cq_timing_part(2)
    finally:
        fc.cq_timing_enable(False)


@pytest.mark.parametrize("prec,bar", [("bf16x3", 2e-5), ("tf32x3", 1e-5)])
def test_direct_mixed_full_size_sampled(fc, prec, bar):
    """The 2D 511x511, N = 8192 precision workload (BE, alpha = (0.2, 0.8), m = 0.45) in the
    configuration the benchmark times; the four lowest and eight seeded sine modes are
    recomputed by the oracle's FP64 direct scheme (measured 3.3e-6 BF16x3, 1.3e-6 TF32x3)."""
    from oracle import spatial as OSP
    p, G0 = ci.workload("prec_2d_m511")
    got, st = _solve(fc, p, G0, fc.CQ_BF16X3 if prec == "bf16x3" else fc.CQ_TF32X3)
    assert st == fc.CQ_OK
    nm = p.M ** p.dim
    sample = np.unique(np.concatenate([[0, 1, p.M, p.M + 1], ci.sample_indices(nm, 8, ci.SEED_BASE + 41)]))
    lam = OSP.mode_eigenvalues(p.M, p.dim)[sample]
    ref = OS.solve_modal(p, lam, OSP.to_modal(G0, p.M, p.dim)[:, sample])[p.N]
    gm = OSP.to_modal(got, p.M, p.dim)[:, sample]
    errs = [float(np.linalg.norm(gm[s] - ref[s]) / np.linalg.norm(ref[s])) for s in range(2)]
    print("mixed direct full size %s: rel L2 errors over %d modes %.3e %.3e" % (prec, len(sample), errs[0], errs[1]))
    assert max(errs) <= bar
