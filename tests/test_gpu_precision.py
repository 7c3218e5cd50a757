"""GPU precision forms against the FP64 oracle (``-m gpu``).

FP32 fast solve (prec = CQ_F32): FP32 history-part states and sums, FP64 tables and
per-mode step matrices, FP64 2x2 step when |a| > 10. Error sources (u = 2^-24):
- a weight rounded to FP32 is a fixed relative error that every step repeats; for the
  window weights (d_1 ~ beta tau^-beta) this acts like an extra reaction term of size
  (a + lambda) |d_1| u and was the largest error (5e-5 on the full workload), so the window
  weights are double-float;
- the ratios r_j of the slowest quarter of the nodes are double-float, the others FP32:
  a rounded ratio near 1 perturbs the geometric weights by up to (u/2) / (1 - r_j) relative,
  < 2e-7 for 1 - r_j > 0.15;
- each history part Y_j is advanced with one FP32 rounding per step; over its memory of
  ~1/(1 - r_j) steps these add up to about u / sqrt(1 - r_j) relative to |Y_j|;
- the levels are FP32 in the ring (node inputs, window terms) and double-float in the
  step and the d_1 term: u per level and step.
These are random in sign and add up over the N steps like a random walk, to ~1e-6 at
N = 8192. Bars: relative L2 error <= 5e-6 per state on the small cases and on the full
2D 511x511, N = 8192 workload (measured <= 1.8e-6; printed).
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


F32_CASES = [
    ("be_1d_m0.3", ci.Problem(0.3, 0.7, 0.3, 1.0, 1024, 1, 63, ci.BE, ci.FAST, 64, 0, 2)),
    ("bdf2_1d_m0.45", ci.Problem(0.2, 0.8, 0.45, 1.0, 2000, 1, 127, ci.BDF2, ci.FAST, 16, 64, 17)),
    ("bdf2_2d_m0.7", ci.Problem(0.4, 0.6, 0.7, 1.0, 600, 2, 23, ci.BDF2, ci.FAST, 12, 36, 15)),
    ("bdf2_1d_m0.48_solve64", ci.Problem(0.5, 0.7, 0.48, 0.5, 800, 1, 31, ci.BDF2, ci.FAST, 16, 48, 17)),
    ("be_2d_np128", ci.Problem(0.6, 0.3, 0.2, 1.0, 1500, 2, 15, ci.BE, ci.FAST, 128, 0, 2)),
    ("bdf2_1d_np5", ci.Problem(0.7, 0.4, 0.6, 1.0, 300, 1, 9, ci.BDF2, ci.FAST, 2, 3, 5)),
    ("be_3d", ci.Problem(0.4, 0.7, 0.3, 1.0, 400, 3, 11, ci.BE, ci.FAST, 64, 0, 2)),
    ("bdf2_2d_ns32_max_window", ci.Problem(0.35, 0.55, 0.4, 1.0, 700, 2, 13, ci.BDF2, ci.FAST, 16, 48, 32)),
    ("bdf2_1d_ns3_min_window", ci.Problem(0.45, 0.65, 0.35, 1.0, 500, 1, 33, ci.BDF2, ci.FAST, 8, 24, 3)),
]


@pytest.mark.parametrize("name,p", F32_CASES, ids=[c[0] for c in F32_CASES])
def test_fast_f32_against_fp64_oracle(fc, name, p):
    G0 = ci.g0_uniform(p.M, p.dim, 17) * 2.0 ** -200          # exercises the per-mode rescaling
    got, st = _solve(fc, p, G0, fc.CQ_F32)
    assert st == fc.CQ_OK
    ref = OS.solve(p, G0)
    errs = [np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s]) for s in range(2)]
    print("f32 %s rel L2 errors %.3e %.3e" % (name, errs[0], errs[1]))
    assert max(errs) <= 5e-6


@pytest.mark.parametrize("alpha", [(0.2, 0.8), (0.8, 0.8)])
def test_fast_f32_full_size_sampled(fc, alpha):
    """The 2D 511x511, N = 8192 precision workload (BE, m = 0.45, Np = 128) in its fast form,
    in the launch configuration the benchmark times; the four lowest and eight seeded sine
    modes are recomputed by the oracle's FP64 fast scheme."""
    from oracle import spatial as OSP
    p, G0 = ci.workload("prec_2d_m511")
    p = p.replace(form=ci.FAST, alpha1=alpha[0], alpha2=alpha[1])
    got, st = _solve(fc, p, G0, fc.CQ_F32)
    assert st == fc.CQ_OK
    nm = p.M ** p.dim
    sample = np.unique(np.concatenate([[0, 1, p.M, p.M + 1], ci.sample_indices(nm, 8, ci.SEED_BASE + 42)]))
    lam = OSP.mode_eigenvalues(p.M, p.dim)[sample]
    ref = OS.solve_modal(p, lam, OSP.to_modal(G0, p.M, p.dim)[:, sample])[p.N]
    gm = OSP.to_modal(got, p.M, p.dim)[:, sample]
    errs = [float(np.linalg.norm(gm[s] - ref[s]) / np.linalg.norm(ref[s])) for s in range(2)]
    print("f32 fast full size %s: rel L2 errors over %d modes %.3e %.3e" % (alpha, len(sample), errs[0], errs[1]))
    assert max(errs) <= 5e-6


def test_fast_f32_rejected_where_unsupported(fc):
    p = ci.Problem(0.3, 0.7, 0.3, 1.0, 64, 1, 15, ci.BE, ci.FAST, 200, 0, 2)   # np > 128
    cp = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                    prec=fc.CQ_F32)
    g0 = torch.zeros((2, 15), dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.fp2s_solve(cp, g0, g0, None), "cuda")
    with pytest.raises(fc.CQError) as e:
        fc.fp2s_solve(cp, g0, torch.empty_like(g0), ws)
    assert e.value.status == fc.CQ_EUNSUPPORTED
    cd = fc.problem(0.3, 0.7, 0.3, 1.0, 64, 1, 15, fc.CQ_BE, fc.CQ_DIRECT, prec=fc.CQ_F32)
    with pytest.raises(fc.CQError):
        fc.fp2s_solve(cd, g0, g0, None)


@pytest.mark.parametrize("scheme,beta,np1,np2,ns,ndof,N", [(2, 0.6, 16, 64, 17, 1001, 300), (1, 0.3, 64, 0, 2, 7, 250),
                                                          (2, 0.45, 8, 12, 5, 4096, 120)])
def test_history_fast_f32_stream(fc, scheme, beta, np1, np2, ns, ndof, N):
    """Streaming FP32 fast history against the oracle's FP64 fast history. Per element the
    error is bounded by 2e-5 of sum_i |d_i| |G^{n-i}| (FP32 levels, states and sums)."""
    from oracle import history as OH
    from oracle import weights as OW
    tau = 1.0 / N
    G = ci.rng(9).standard_normal((N + 1, ndof))
    Gd = torch.tensor(G, dtype=torch.float64, device="cuda")
    H = torch.empty(ndof, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_fast(scheme, beta, tau, np1, np2, ns, ndof, 1, None, None, prec=fc.CQ_F32),
                      "cuda")
    ref_h = OH.FastHistoryBE(beta, tau, np1, ndof) if scheme == 1 else OH.FastHistorySBD(beta, tau, np1, np2, ns,
                                                                                          ndof)
    d = OW.weights(scheme, beta, tau, N)
    worst = 0.0
    for n in range(1, N + 1):
        fc.cq_history_fast(scheme, beta, tau, np1, np2, ns, ndof, n, Gd[n - 1], H, ws, prec=fc.CQ_F32)
        torch.cuda.synchronize()
        got = H.cpu().numpy()
        ref = ref_h(n, G)
        scale = np.abs(d[n - 1:0:-1]) @ np.abs(G[1:n]) if n >= 2 else np.zeros(ndof)
        err = np.abs(got - ref)
        assert np.all(err <= 2e-5 * scale + 1e-300), n
        if n >= 2:
            worst = max(worst, float(np.max(err / (scale + 1e-300))))
    print("f32 stream history: max |err| / sum|d||G| = %.3e" % worst)


def test_fp32_forms_report_range_overflow(fc):
    """m = 0.49 (a = -25.5) on a 2D grid: the lowest mode grows by about 2^550 by t = 1/4, far
    beyond the FP32 range after its single power-of-two prescale. The FP32 fast solve and the
    mixed-precision direct solve report CQ_ENONFINITE; the FP64 solve stays finite."""
    G0 = ci.g0_uniform(15, 2, 9)
    fast = ci.Problem(0.4, 0.6, 0.49, 0.25, 256, 2, 15, ci.BDF2, ci.FAST, 16, 64, 17)
    direct = fast.replace(form=ci.DIRECT)
    g64, st64 = _solve(fc, fast, G0, fc.CQ_F64)
    assert st64 == fc.CQ_OK and np.all(np.isfinite(g64))
    assert np.log2(np.max(np.abs(g64))) > 300
    _, st32 = _solve(fc, fast, G0, fc.CQ_F32)
    assert st32 == fc.CQ_ENONFINITE
    _, stmx = _solve(fc, direct, G0, fc.CQ_BF16X3)
    assert stmx == fc.CQ_ENONFINITE
