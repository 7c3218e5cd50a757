"""GPU parity: every entry point of the C ABI against the FP64 CPU oracle on the
same seeded inputs (``-m gpu``).

Tolerances (FP64 on both sides, same algorithm, different rounding order):
* weights: relative 1e-12; Gauss-Jacobi nodes and the ratios r_j: absolute 2e-15 / 4e-15;
  Gauss-Jacobi weights and the coefficients c_j: relative 1e-11 (a node error of 1e-16
  moves the tiny end weights by up to ~1e-12 relative);
* histories: |gpu - oracle| <= 1e-12 * sum_i |d_i| |G^{n-i}| element by element,
  i.e. relative to the condition of the sum, not to its possibly cancelled value;
* solves: relative L2 error <= 1e-12 per state and max element error <= 1e-11 * max|ref|.
"""
import numpy as np
import pytest

import cq_inputs as ci
from oracle import history as OH
from oracle import quadrature as OQ
from oracle import scheme as OS
from oracle import spatial as OSP
from oracle import weights as OW

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_05128_gb300 as pkg
    pkg.build()
    return pkg.load()


DEV = "cuda"


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# ---------------------------------------------------------------- weights / rules
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("beta,tau,n", [(0.3, 1e-3, 0), (0.7, 1e-3, 1), (0.6, 1 / 4096, 4096), (0.2, 1 / 8192, 8192),
                                        (0.5, 0.05, 1000), (0.625, 1 / 2000, 20000)])
def test_weights(fc, scheme, beta, tau, n):
    w = torch.empty(n + 1, dtype=torch.float64, device=DEV)
    fc.cq_weights(scheme, beta, tau, n, w)
    got = _np(w)
    ref = OW.weights(scheme, beta, tau, n)
    scale = np.max(np.abs(ref))
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-15 * scale)


@pytest.mark.parametrize("n,a,b", [(1, 0.3, 0.7), (7, 0.6, 0.4), (32, 0.4, 1.2), (64, 0.2, 1.6), (80, 0.75, 0.25),
                                   (128, 0.7, 0.3), (181, 0.5, 1.0), (256, 0.8, 0.4)])
def test_gauss_jacobi(fc, n, a, b):
    x = torch.empty(n, dtype=torch.float64, device=DEV)
    lw = torch.empty(n, dtype=torch.float64, device=DEV)
    fc.cq_gauss_jacobi(n, a, b, x, lw)
    xr, lr = OQ.gauss_jacobi(n, a, b)
    assert np.max(np.abs(_np(x) - xr)) < 2e-15
    assert np.max(np.abs(_np(lw) / lr - 1.0)) < 1e-11


@pytest.mark.parametrize("scheme,beta,tau,np1,np2,ns", [(1, 0.7, 1 / 1024, 64, 0, 2), (1, 0.3, 1e-3, 181, 0, 2),
                                                        (2, 0.6, 1 / 4096, 16, 64, 17), (2, 0.4, 1 / 4096, 16, 64, 17),
                                                        (2, 0.8, 1e-3, 41, 41, 15), (2, 0.2, 0.01, 5, 9, 3)])
def test_fast_coeffs(fc, scheme, beta, tau, np1, np2, ns):
    npt = np1 + (np2 if scheme == 2 else 0)
    coef = torch.empty(2 * npt, dtype=torch.float64, device=DEV)
    ws = fc.workspace(fc.cq_fast_coeffs(scheme, beta, tau, np1, np2, ns, None), DEV)
    fc.cq_fast_coeffs(scheme, beta, tau, np1, np2, ns, coef, ws)
    got = _np(coef)
    if scheme == 1:
        c = OQ.be_fast_coefficients(beta, tau, np1)
        r_ref, c_ref = c.r, c.w
    else:
        c = OQ.sbd_fast_coefficients(beta, tau, np1, np2, ns)
        r_ref, c_ref = np.concatenate([c.r1, c.r2]), np.concatenate([c.q1, c.q2])
    # r = (s+1)/2 or (s+1)/(s+5) inherits the absolute accuracy of the node s (its
    # relative accuracy degrades near s = -1); c carries r^(Ns-3) on top.
    assert np.max(np.abs(got[:npt] - r_ref)) < 4e-15
    assert np.max(np.abs(got[npt:] / c_ref - 1.0)) < 1e-11


# ---------------------------------------------------------------- histories
def _abs_scale(d, G, n):
    if n < 2:
        return np.zeros(G.shape[1])
    return np.abs(d[n - 1:0:-1]) @ np.abs(G[1:n])


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("ndof,n_lo,n_hi,ld_extra", [(1, 1, 40, 0), (5, 2, 37, 1), (127, 1, 300, 0),
                                                     (1000, 17, 333, 3), (4097, 250, 301, 0), (256, 1, 2, 0)])
def test_history_direct(fc, scheme, ndof, n_lo, n_hi, ld_extra):
    beta, tau = 0.37, 1.0 / 500
    ld = ndof + ld_extra
    G = np.zeros((n_hi, ld))
    G[:, :ndof] = ci.rng(5).standard_normal((n_hi, ndof))
    Gd = _t(G)
    H = torch.full(((n_hi - n_lo), ld), np.nan, dtype=torch.float64, device=DEV)
    ws = fc.workspace(fc.cq_history_direct(scheme, beta, tau, ndof, n_lo, n_hi, None, ld, None, ld), DEV)
    fc.cq_history_direct(scheme, beta, tau, ndof, n_lo, n_hi, Gd, ld, H, ld, ws)
    got = _np(H)[:, :ndof]
    d = OW.weights(scheme, beta, tau, n_hi)
    ref = OH.history_direct_all(d, G[:, :ndof], n_lo, n_hi)
    scale = np.stack([_abs_scale(d, G[:, :ndof], n) for n in range(n_lo, n_hi)])
    assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300)
    if ld_extra:                                    # padding columns untouched
        assert np.all(np.isnan(_np(H)[:, ndof:]))


@pytest.mark.parametrize("prec", [0, 4], ids=["f64", "df64"])
@pytest.mark.parametrize("scheme,beta,np1,np2,ns,ndof,N", [(1, 0.7, 24, 0, 2, 131, 400), (1, 0.3, 64, 0, 2, 2, 300),
                                                          (2, 0.6, 16, 64, 17, 257, 300), (2, 0.4, 8, 12, 5, 1, 120),
                                                          (2, 0.8, 31, 31, 15, 64, 250)])
def test_history_fast(fc, scheme, beta, np1, np2, ns, ndof, N, prec):
    """FP64 and the double-float form (CQ_DF64) against the oracle at the FP64 bar."""
    tau = 1.0 / N
    G = ci.rng(7).standard_normal((N + 1, ndof))
    H = torch.empty(ndof, dtype=torch.float64, device=DEV)
    ws = fc.workspace(fc.cq_history_fast(scheme, beta, tau, np1, np2, ns, ndof, 1, None, None, prec=prec), DEV)
    if scheme == 1:
        ref_h = OH.FastHistoryBE(beta, tau, np1, ndof)
    else:
        ref_h = OH.FastHistorySBD(beta, tau, np1, np2, ns, ndof)
    d = OW.weights(scheme, beta, tau, N)
    Gd = _t(G)
    for n in range(1, N + 1):
        fc.cq_history_fast(scheme, beta, tau, np1, np2, ns, ndof, n, Gd[n - 1], H, ws, prec=prec)
        got = _np(H)
        ref = ref_h(n, G)
        scale = _abs_scale(d, G, n)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300), n


# ---------------------------------------------------------------- solves
def _cproblem(fc, p, flags=0):
    return fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                      flags=flags)


def _solve_gpu(fc, p, G0):
    cp = _cproblem(fc, p)
    g0 = _t(G0)
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), DEV)
    st = fc.fp2s_solve(cp, g0, gN, ws, check=False)
    return _np(gN), st


SOLVES = [
    ("be1d_m63", None),                                                                  # the 1D BE direct workload
    ("be1d_m63_fast", ci.Problem(0.3, 0.7, 0.4, 1.0, 1024, 1, 63, ci.BE, ci.FAST, 64, 0, 2)),
    ("bdf2_1d", ci.Problem(0.4, 0.6, 0.3, 1.0, 700, 1, 45, ci.BDF2, ci.DIRECT)),
    ("bdf2_1d_fast", ci.Problem(0.4, 0.6, 0.3, 1.0, 700, 1, 45, ci.BDF2, ci.FAST, 16, 48, 17)),
    ("be2d_fast", ci.Problem(0.25, 0.55, 0.7, 0.5, 333, 2, 21, ci.BE, ci.FAST, 40, 0, 2)),
    ("bdf2_2d", ci.Problem(0.2, 0.8, 0.0, 1.0, 257, 2, 19, ci.BDF2, ci.DIRECT)),
    ("bdf2_2d_fast", ci.Problem(0.2, 0.8, 0.45, 1.0, 257, 2, 19, ci.BDF2, ci.FAST, 9, 23, 7)),
    ("tiny", ci.Problem(0.5, 0.5, 0.6, 1.0, 3, 1, 1, ci.BDF2, ci.FAST, 2, 2, 3)),
    ("one_step", ci.Problem(0.5, 0.5, 0.6, 1.0, 1, 2, 3, ci.BE, ci.DIRECT)),
    ("be3d", ci.Problem(0.35, 0.7, 0.4, 1.0, 120, 3, 9, ci.BE, ci.DIRECT)),
    ("bdf2_3d_fast", ci.Problem(0.3, 0.6, 0.65, 1.0, 150, 3, 11, ci.BDF2, ci.FAST, 12, 30, 9)),
    ("be3d_fast_ragged", ci.Problem(0.6, 0.45, 0.3, 0.5, 77, 3, 13, ci.BE, ci.FAST, 40, 0, 2)),
    # mode counts on both sides of the lane-split thresholds of the direct solve (32, 16, 8, 4
    # lanes per mode below 4864, 9728, 19456, 38912 modes) and of the fast solve (a warp per
    # mode below 9728 modes)
    ("direct_lp16", ci.Problem(0.3, 0.7, 0.4, 1.0, 30, 2, 70, ci.BE, ci.DIRECT)),
    ("direct_lp8", ci.Problem(0.5, 0.6, 0.6, 1.0, 25, 2, 100, ci.BDF2, ci.DIRECT)),
    ("direct_lp4", ci.Problem(0.3, 0.7, 0.4, 1.0, 20, 2, 150, ci.BE, ci.DIRECT)),
    ("direct_lp1", ci.Problem(0.3, 0.7, 0.4, 1.0, 12, 2, 200, ci.BDF2, ci.DIRECT)),
    ("fast_warp_per_mode", ci.Problem(0.4, 0.6, 0.3, 1.0, 60, 2, 98, ci.BDF2, ci.FAST, 16, 64, 17)),
    ("fast_16_per_warp", ci.Problem(0.4, 0.6, 0.3, 1.0, 60, 2, 99, ci.BDF2, ci.FAST, 16, 64, 17)),
]


@pytest.mark.parametrize("name,p", SOLVES, ids=[s[0] for s in SOLVES])
def test_fp2s_solve(fc, name, p):
    if p is None:
        p, G0 = ci.workload(name)
    else:
        G0 = ci.g0_uniform(p.M, p.dim, 99)
    got, st = _solve_gpu(fc, p, G0)
    assert st == fc.CQ_OK
    ref = OS.solve(p, G0)
    for s in range(2):
        assert np.linalg.norm(got[s] - ref[s]) <= 1e-12 * np.linalg.norm(ref[s])
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("p", [ci.Problem(0.3, 0.6, 0.2, 1.0, 90, 1, 31, ci.BE, ci.DIRECT),
                               ci.Problem(0.3, 0.6, 0.2, 1.0, 90, 2, 7, ci.BDF2, ci.FAST, 6, 10, 5),
                               ci.Problem(0.3, 0.6, 0.2, 1.0, 40, 3, 5, ci.BDF2, ci.DIRECT)])
def test_fp2s_step_levels(fc, p):
    G0 = ci.g0_uniform(p.M, p.dim, 3)
    _, g_ref = OS.solve(p, G0, all_levels=True)
    cp = _cproblem(fc, p)
    g0 = _t(G0)
    ws = fc.workspace(fc.fp2s_init(cp, g0, None), DEV)
    fc.fp2s_init(cp, g0, ws)
    out = torch.empty_like(g0)
    modal = torch.empty_like(g0)
    for n in range(1, p.N + 1):
        fc.fp2s_step(cp, n, ws, out if n % 7 == 0 or n == p.N else None)
        fc.fp2s_modal(cp, ws, modal)
        gm = _np(modal)
        assert np.max(np.abs(gm - g_ref[n])) <= 1e-11 * np.max(np.abs(g_ref[n])), n
        if n % 7 == 0 or n == p.N:
            phys = OSP.to_physical(g_ref[n], p.M, p.dim)
            assert np.max(np.abs(_np(out) - phys)) <= 1e-11 * np.max(np.abs(phys))
    assert fc.fp2s_status(cp, ws) == fc.CQ_OK


def test_nonfinite_reported(fc):
    p = ci.Problem(0.4, 0.6, 0.49, 1.0, 64, 1, 7, ci.BE, ci.DIRECT)
    G0 = ci.g0_uniform(7, 1, 1)
    G0[0, 3] = np.nan
    _, st = _solve_gpu(fc, p, G0)
    assert st == fc.CQ_ENONFINITE


# ---------------------------------------------------------------- full-size workload, sampled modes
@pytest.mark.parametrize("form", [ci.FAST, ci.DIRECT])
def test_bdf2_2d_m255_sampled_modes(fc, form):
    """The 2D 255x255 BDF2 workload (N = 4096, m = 0.49) at full size in the launch
    configuration the benchmark times. G0 is scaled by 2^-1000 so that the mode that
    grows like e^(1096 t) stays finite (the scheme is linear, so the arithmetic is the
    same up to the exact power-of-two factor). 48 seeded modes plus the 4 lowest are
    recomputed by the oracle one by one and compared in the sine basis."""
    p, G0 = ci.workload("bdf2_2d_m255")
    p = p.replace(form=form)
    G0 = G0 * 2.0 ** -1000
    got, st = _solve_gpu(fc, p, G0)
    assert st == fc.CQ_OK
    ghat = OSP.to_modal(got, p.M, p.dim)
    nm = p.M ** 2
    sample = np.unique(np.concatenate([[0, 1, p.M, p.M + 1], ci.sample_indices(nm, 48, ci.SEED_BASE + 11)]))
    lam = OSP.mode_eigenvalues(p.M, p.dim)[sample]
    g0 = OSP.to_modal(G0, p.M, p.dim)[:, sample]
    ref = OS.solve_modal(p, lam, g0)[p.N]
    err = np.abs(ghat[:, sample] - ref)
    # modal values of the GPU result pass through two DSTs (to physical and back):
    # each adds rounding of order eps * sqrt(nm) * max|g| to every coefficient.
    floor = 1e-13 * np.max(np.abs(ref))
    assert np.all(err <= 1e-10 * np.abs(ref) + floor), np.max(err / (np.abs(ref) + floor))
