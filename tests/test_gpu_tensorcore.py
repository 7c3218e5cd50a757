"""Tensor-core direct history (prec = CQ_BF16X3) against the FP64 oracle (``-m gpu``).

Error bound, from the arithmetic: BF16 keeps 8 significant bits (unit roundoff
2^-8), so hi = bf16(x) and lo = bf16(x - hi) leave |x - hi - lo| <= 2^-16 |x|;
products of BF16 numbers are exact in FP32; the dropped lo*lo term is <= 2^-16 |a||b|.
The accumulator rounds toward zero once per MMA instruction (K = 16 levels, three
products) within a chunk of 128 levels: 24 roundings of <= 2^-23 of the chunk's sum of
absolute terms; the chunks are added to FP32 running sums with round-to-nearest
(ceil(K / 128) roundings of <= 2^-24). So element by element
    |H_tc - H| <= (3 * 2^-16 + 24 * 2^-23 + ceil(K / 128) * 2^-24) * sum_i |d_i| |G^{n-i}|.
An accumulation over all K levels in the truncating accumulator (3 K / 16 roundings)
would exceed it. The measured errors are printed beside the bound.
"""
import numpy as np
import pytest

import cq_inputs as ci
from oracle import history as OH
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


def _bound(K):
    return 3 * 2.0 ** -16 + 24 * 2.0 ** -23 + (-(-K // 128)) * 2.0 ** -24


def _abs_scale(d, G, n):
    if n < 2:
        return np.zeros(G.shape[1])
    return np.abs(d[n - 1:0:-1]) @ np.abs(G[1:n])


CASES = [(1, 1, 2, 0), (1, 1, 3, 0), (100, 1, 65, 0), (300, 1, 130, 5), (257, 2, 300, 0),
         (1000, 50, 200, 3), (513, 120, 400, 0), (2048, 1, 700, 0)]


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("ndof,n_lo,n_hi,ld_extra", CASES)
def test_bf16x3_history_small(fc, scheme, ndof, n_lo, n_hi, ld_extra):
    beta, tau = 0.45, 1.0 / 700
    ld = ndof + ld_extra
    G = np.zeros((n_hi, ld))
    G[:, :ndof] = ci.rng(41).standard_normal((n_hi, ndof))
    Gd = torch.tensor(G, dtype=torch.float64, device="cuda")
    H = torch.full((n_hi - n_lo, ld), np.nan, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_direct(scheme, beta, tau, ndof, n_lo, n_hi, None, ld, None, ld,
                                           prec=fc.CQ_BF16X3), "cuda")
    fc.cq_history_direct(scheme, beta, tau, ndof, n_lo, n_hi, Gd, ld, H, ld, ws, prec=fc.CQ_BF16X3)
    torch.cuda.synchronize()
    got = H.cpu().numpy()
    d = OW.weights(scheme, beta, tau, n_hi)
    ref = OH.history_direct_all(d, G[:, :ndof], n_lo, n_hi)
    scale = np.stack([_abs_scale(d, G[:, :ndof], n) for n in range(n_lo, n_hi)])
    err = np.abs(got[:, :ndof] - ref)
    ratio = float(np.max(err / (scale + 1e-300)))
    print("bf16x3 ndof=%d rows=[%d,%d): max |err| / sum|d||G| = %.3e (bound %.3e)"
          % (ndof, n_lo, n_hi, ratio, _bound(n_hi)))
    assert np.all(err <= _bound(n_hi) * scale + 1e-300)
    if ld_extra:
        assert np.all(np.isnan(got[:, ndof:]))


def test_bf16x3_history_full_size_sampled(fc):
    """The 2D 511x511 contraction at its full size (522,242 DOFs, levels up to 8192) in
    the launch configuration the benchmark times, for the last 193 steps; 24 whole DOF
    columns are recomputed by the oracle and checked against the bound."""
    ndof, n_lo, n_hi = 2 * 511 * 511, 8000, 8193
    beta, tau = 0.8, 1.0 / 8192
    gen = torch.Generator(device="cuda")
    gen.manual_seed(ci.SEED_BASE + 5)
    G = torch.randn(n_hi, ndof, dtype=torch.float64, device="cuda", generator=gen)
    H = torch.empty(n_hi - n_lo, ndof, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, None, ndof, None, ndof,
                                           prec=fc.CQ_BF16X3), "cuda")
    fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, G, ndof, H, ndof, ws, prec=fc.CQ_BF16X3)
    torch.cuda.synchronize()
    cols = np.concatenate([[0, ndof - 1], ci.sample_indices(ndof, 22, ci.SEED_BASE + 6)])
    idx = torch.tensor(cols, device="cuda")
    Gc = G[:, idx].cpu().numpy()
    Hc = H[:, idx].cpu().numpy()
    del G, H, ws
    torch.cuda.empty_cache()
    d = OW.weights(1, beta, tau, n_hi)
    ref = OH.history_direct_all(d, Gc, n_lo, n_hi)
    scale = np.stack([_abs_scale(d, Gc, n) for n in range(n_lo, n_hi)])
    err = np.abs(Hc - ref)
    print("bf16x3 full size: max |err| / sum|d||G| = %.3e" % float(np.max(err / scale)))
    assert np.all(err <= _bound(n_hi) * scale)


def test_bf16x3_history_more_dof_tiles_than_grid_rows(fc):
    """2.2 M DOFs: more 32-DOF tiles of the split-transpose than a grid has rows (65,535), so
    its CTAs take further DOF tiles in turn; sampled columns from the first and the last
    tiles are checked against the oracle."""
    ndof, n_lo, n_hi = 2_200_000, 1, 70
    beta, tau = 0.6, 1.0 / 64
    gen = torch.Generator(device="cuda")
    gen.manual_seed(ci.SEED_BASE + 8)
    G = torch.randn(n_hi, ndof, dtype=torch.float64, device="cuda", generator=gen)
    H = torch.empty(n_hi - n_lo, ndof, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_direct(2, beta, tau, ndof, n_lo, n_hi, None, ndof, None, ndof,
                                           prec=fc.CQ_BF16X3), "cuda")
    fc.cq_history_direct(2, beta, tau, ndof, n_lo, n_hi, G, ndof, H, ndof, ws, prec=fc.CQ_BF16X3)
    torch.cuda.synchronize()
    cols = np.concatenate([[0, 31, 32 * 65535, 32 * 65535 + 7, ndof - 1],
                           ci.sample_indices(ndof, 27, ci.SEED_BASE + 9)])
    idx = torch.tensor(cols, device="cuda")
    Gc = G[:, idx].cpu().numpy()
    Hc = H[:, idx].cpu().numpy()
    del G, H, ws
    torch.cuda.empty_cache()
    d = OW.weights(2, beta, tau, n_hi)
    ref = OH.history_direct_all(d, Gc, n_lo, n_hi)
    scale = np.stack([_abs_scale(d, Gc, n) for n in range(n_lo, n_hi)])
    assert np.all(np.abs(Hc - ref) <= _bound(n_hi) * scale + 1e-300)


def _bound_tf32(K):
    """TF32x3: each split operand keeps 22 bits (<= 2^-22 relative) and the dropped lo*lo
    term is <= 2^-22, so the products carry <= 4 * 2^-22; the accumulator rounds toward
    zero once per K = 8 instruction and product within a 32-level chunk (12 roundings,
    <= 2^-23 each, relative to the chunk's sum of |terms|), and the chunks are summed in
    FP32 with round-to-nearest (<= ceil(K / 32) roundings of 2^-24)."""
    return 4 * 2.0 ** -22 + 12 * 2.0 ** -23 + (-(-K // 32)) * 2.0 ** -24


def _run_history(fc, prec, scheme, beta, tau, G, ndof, n_lo, n_hi, ld):
    Gd = torch.tensor(G, dtype=torch.float64, device="cuda")
    H = torch.full((n_hi - n_lo, ld), np.nan, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_direct(scheme, beta, tau, ndof, n_lo, n_hi, None, ld, None, ld, prec=prec), "cuda")
    fc.cq_history_direct(scheme, beta, tau, ndof, n_lo, n_hi, Gd, ld, H, ld, ws, prec=prec)
    torch.cuda.synchronize()
    return H.cpu().numpy()


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("ndof,n_lo,n_hi,ld_extra", CASES)
def test_tf32x3_history_small(fc, scheme, ndof, n_lo, n_hi, ld_extra):
    beta, tau = 0.45, 1.0 / 700
    ld = ndof + ld_extra
    G = np.zeros((n_hi, ld))
    G[:, :ndof] = ci.rng(41).standard_normal((n_hi, ndof))
    got = _run_history(fc, fc.CQ_TF32X3, scheme, beta, tau, G, ndof, n_lo, n_hi, ld)
    d = OW.weights(scheme, beta, tau, n_hi)
    ref = OH.history_direct_all(d, G[:, :ndof], n_lo, n_hi)
    scale = np.stack([_abs_scale(d, G[:, :ndof], n) for n in range(n_lo, n_hi)])
    err = np.abs(got[:, :ndof] - ref)
    ratio = float(np.max(err / (scale + 1e-300)))
    print("tf32x3 ndof=%d rows=[%d,%d): max |err| / sum|d||G| = %.3e (bound %.3e)"
          % (ndof, n_lo, n_hi, ratio, _bound_tf32(n_hi)))
    assert np.all(err <= _bound_tf32(n_hi) * scale + 1e-300)
    if ld_extra:
        assert np.all(np.isnan(got[:, ndof:]))


def test_tf32x3_more_accurate_than_bf16x3(fc):
    """Same data through both forms: the TF32 split error is 2^6 times smaller, so the
    TF32x3 history is at least 8x closer to the FP64 oracle in the max norm."""
    ndof, n_lo, n_hi, beta, tau = 1500, 1, 900, 0.7, 1.0 / 900
    G = ci.rng(43).standard_normal((n_hi, ndof))
    d = OW.weights(1, beta, tau, n_hi)
    ref = OH.history_direct_all(d, G, n_lo, n_hi)
    e_b = np.max(np.abs(_run_history(fc, fc.CQ_BF16X3, 1, beta, tau, G, ndof, n_lo, n_hi, ndof) - ref))
    e_t = np.max(np.abs(_run_history(fc, fc.CQ_TF32X3, 1, beta, tau, G, ndof, n_lo, n_hi, ndof) - ref))
    print("max error: bf16x3 %.3e, tf32x3 %.3e" % (e_b, e_t))
    assert e_t * 8 <= e_b


def test_tf32x3_history_full_size_sampled(fc):
    """The 2D 511x511 contraction at its full size in the TF32x3 form, last 193 steps, 24
    whole DOF columns recomputed by the oracle."""
    ndof, n_lo, n_hi = 2 * 511 * 511, 8000, 8193
    beta, tau = 0.8, 1.0 / 8192
    gen = torch.Generator(device="cuda")
    gen.manual_seed(ci.SEED_BASE + 5)
    G = torch.randn(n_hi, ndof, dtype=torch.float64, device="cuda", generator=gen)
    H = torch.empty(n_hi - n_lo, ndof, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, None, ndof, None, ndof,
                                           prec=fc.CQ_TF32X3), "cuda")
    fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, G, ndof, H, ndof, ws, prec=fc.CQ_TF32X3)
    torch.cuda.synchronize()
    cols = np.concatenate([[0, ndof - 1], ci.sample_indices(ndof, 22, ci.SEED_BASE + 6)])
    idx = torch.tensor(cols, device="cuda")
    Gc = G[:, idx].cpu().numpy()
    Hc = H[:, idx].cpu().numpy()
    del G, H, ws
    torch.cuda.empty_cache()
    d = OW.weights(1, beta, tau, n_hi)
    ref = OH.history_direct_all(d, Gc, n_lo, n_hi)
    scale = np.stack([_abs_scale(d, Gc, n) for n in range(n_lo, n_hi)])
    err = np.abs(Hc - ref)
    print("tf32x3 full size: max |err| / sum|d||G| = %.3e" % float(np.max(err / scale)))
    assert np.all(err <= _bound_tf32(n_hi) * scale)
