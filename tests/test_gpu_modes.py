"""Solves in the sine basis (fp2s_solve_modes, ``-m gpu``): FP64 parity of the full-size
workload without transforms, and ranges of modes solved in separate calls.

In the sine basis of the Dirichlet Laplacian every mode is an independent 2x2 system
(Eq. 2.1 with A diagonal), so the modal levels of the GPU can be compared with the
oracle's per-mode scheme directly, and a grid's modes can be split into contiguous
shards (one per device) with no exchange between them.
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


def _cp(fc, p, prec=0):
    return fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                      prec=prec)


def _modes(fc, cp, g0m, lo, hi):
    g0 = torch.tensor(np.ascontiguousarray(g0m[:, lo:hi]), dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve_modes(cp, lo, hi, g0, gN, None), "cuda")
    st = fc.fp2s_solve_modes(cp, lo, hi, g0, gN, ws, check=False)
    torch.cuda.synchronize()
    return gN.cpu().numpy(), st


def _rel_per_state(got, ref):
    """Relative L2 error per state (scaled first: the m = 0.49 workload's growing mode
    reaches ~2^581, whose square overflows FP64)."""
    out = []
    for s in range(2):
        sc = np.max(np.abs(ref[s]))
        out.append(float(np.linalg.norm((got[s] - ref[s]) / sc) / np.linalg.norm(ref[s] / sc)))
    return out


@pytest.mark.parametrize("form,prec", [(ci.FAST, 0), (ci.DIRECT, 0), (ci.FAST, 4)],
                         ids=["fast_f64", "direct_f64", "fast_df64"])
def test_bdf2_2d_m255_modal_parity(fc, form, prec):
    """The 2D 255x255 BDF2 workload (N = 4096, m = 0.49, G0 x 2^-1000) over all 65,025 modes
    in the launch configuration of the benchmark, compared in the sine basis with the oracle's
    FP64 scheme (same form, same tables) on the 4 lowest and 60 seeded modes, with no
    transform on either side: relative L2 error per state <= 1e-12 over the decaying modes.
    Three sampled modes grow (a = -25.5): (1,1) like e^(1096 t), (1,2) and (2,1) like
    e^(2.7 t). Their g^N is a high power of a per-step amplification that both sides form
    from FP64 coefficients, so a relative error of one unit in the last place of a
    coefficient becomes many units in g^N. The test measures that conditioning with the
    oracle itself (the largest change of g^N when lambda_k, a or T moves by one ulp) and
    bounds the GPU's error on each growing mode by 4 x it. The double-float fast form
    (CQ_DF64) is held to the same bars."""
    p, G0 = ci.workload("bdf2_2d_m255")
    p = p.replace(form=form)
    g0m = OSP.to_modal(G0 * 2.0 ** -1000, p.M, p.dim)
    nm = p.M ** p.dim
    got, st = _modes(fc, _cp(fc, p, prec), g0m, 0, nm)
    assert st == fc.CQ_OK
    sample = np.unique(np.concatenate([[0, 1, p.M, p.M + 1], ci.sample_indices(nm, 60, ci.SEED_BASE + 12)]))
    lam_all = OSP.mode_eigenvalues(p.M, p.dim)
    growing = np.array([ci.growth_rate(p.alpha1, p.alpha2, p.m, lam_all[k]) > 0.0 for k in sample])
    assert growing.sum() == 3
    calm = sample[~growing]
    ref = OS.solve_modal(p, lam_all[calm], g0m[:, calm])[p.N]
    errs = _rel_per_state(got[:, calm], ref)
    print("modal parity %s%s: rel L2 per state %.3e %.3e over %d decaying modes"
          % ("fast" if form == ci.FAST else "direct", " df64" if prec == 4 else "", errs[0], errs[1], len(calm)))
    assert max(errs) <= 1e-12
    one_ulp = 2.0 ** -52
    for k in sample[growing]:
        lam_k, g0_k = lam_all[[k]], g0m[:, [k]]
        ref_k = OS.solve_modal(p, lam_k, g0_k)[p.N]
        moved = [OS.solve_modal(p, lam_k * (1 + one_ulp), g0_k)[p.N],
                 OS.solve_modal(p, lam_k, g0_k, a=OS.coupling(p.m) * (1 + one_ulp))[p.N],
                 OS.solve_modal(p.replace(T=p.T * (1 + one_ulp)), lam_k, g0_k)[p.N]]
        kappa = max(float(np.max(np.abs(m_ - ref_k)) / np.max(np.abs(ref_k))) for m_ in moved)
        err_k = float(np.max(np.abs(got[:, [k]] - ref_k)) / np.max(np.abs(ref_k)))
        print("  growing mode %d: rel error %.3e, one-ulp conditioning %.3e" % (k, err_k, kappa))
        assert err_k <= 4.0 * kappa


SHARD_CASES = [
    ("fast_f64_2d", ci.Problem(0.4, 0.6, 0.3, 1.0, 300, 2, 255, ci.BDF2, ci.FAST, 16, 48, 17), 0),
    ("direct_f64_2d", ci.Problem(0.3, 0.7, 0.4, 1.0, 200, 2, 283, ci.BE, ci.DIRECT, 0, 0, 0), 0),
    ("fast_f32_2d", ci.Problem(0.2, 0.8, 0.45, 1.0, 400, 2, 127, ci.BE, ci.FAST, 64, 0, 2), 1),
    ("fast_df64_2d", ci.Problem(0.4, 0.6, 0.3, 1.0, 300, 2, 255, ci.BDF2, ci.FAST, 16, 48, 17), 4),
    ("mixed_bf16x3_2d", ci.Problem(0.4, 0.6, 0.3, 1.0, 300, 2, 255, ci.BDF2, ci.DIRECT, 0, 0, 0), 2),
    ("mixed_tf32x3_2d", ci.Problem(0.3, 0.7, 0.4, 1.0, 260, 2, 255, ci.BE, ci.DIRECT, 0, 0, 0), 3),
]


@pytest.mark.parametrize("name,p,prec", SHARD_CASES, ids=[c[0] for c in SHARD_CASES])
def test_two_shards_equal_whole(fc, name, p, prec):
    """The modes split into two contiguous shards at an uneven point, each solved by its own
    call as a device of a two-device run would: concatenated, they equal the whole-range
    solve bit for bit (both shards are large enough to take the same kernel as the whole),
    and the whole range matches the oracle at the form's tolerance."""
    nm = p.M ** p.dim
    g0m = OSP.to_modal(ci.g0_uniform(p.M, p.dim, 29), p.M, p.dim)
    cp = _cp(fc, p, prec)
    whole, st = _modes(fc, cp, g0m, 0, nm)
    assert st == fc.CQ_OK
    cut = nm // 2 + 37
    a, sta = _modes(fc, cp, g0m, 0, cut)
    b, stb = _modes(fc, cp, g0m, cut, nm)
    assert sta == fc.CQ_OK and stb == fc.CQ_OK
    assert np.array_equal(np.concatenate([a, b], axis=1), whole)
    sample = np.unique(np.concatenate([[0, 1, cut - 1, cut, nm - 1], ci.sample_indices(nm, 24, ci.SEED_BASE + 13)]))
    ref = OS.solve_modal(p, OSP.mode_eigenvalues(p.M, p.dim)[sample], g0m[:, sample])[p.N]
    errs = _rel_per_state(whole[:, sample], ref)
    print("shards %s: rel L2 per state vs oracle %.3e %.3e" % (name, *errs))
    assert max(errs) <= (1e-12 if prec in (0, 4) else 2e-5)


def test_single_mode_range(fc):
    """A range of one mode (the last one of the grid), through the few-mode kernels."""
    p = ci.Problem(0.4, 0.6, 0.3, 1.0, 150, 2, 31, ci.BDF2, ci.FAST, 8, 24, 9)
    nm = p.M ** p.dim
    g0m = OSP.to_modal(ci.g0_uniform(p.M, p.dim, 31), p.M, p.dim)
    got, st = _modes(fc, _cp(fc, p), g0m, nm - 1, nm)
    assert st == fc.CQ_OK
    ref = OS.solve_modal(p, OSP.mode_eigenvalues(p.M, p.dim)[nm - 1:], g0m[:, nm - 1:])[p.N]
    assert max(_rel_per_state(got, ref)) <= 1e-12
