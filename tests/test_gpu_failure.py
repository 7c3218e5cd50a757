"""The failure path of the tensor-core kernels, made to run without a fault or a hang.

cq_test_expire_waits(True) makes every tensor-core CTA withhold its first operand load and
bounds the waits between its roles by 10 ms: the MMA thread's wait for that load expires,
the CTA records the timeout, writes NaN to its tiles, drains its loads and frees its tensor
memory. The calls must report it (CQ_ETIMEOUT, or NaN where the history could not be
formed), and after the switch is off the same calls on the same workspaces must give the
oracle's results again: the device stays usable."""
import numpy as np
import pytest

import cq_inputs as ci
from oracle import history as OH
from oracle import scheme as OS
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


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_expired_wait_in_mixed_solve(fc, prec):
    p = ci.Problem(0.3, 0.7, 0.4, 1.0, 300, 1, 63, ci.BE, ci.DIRECT, 0, 0, 0)     # 3 blocks: contractions run
    pr = fc.CQ_BF16X3 if prec == "bf16x3" else fc.CQ_TF32X3
    cp = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, prec=pr)
    G0 = ci.g0_uniform(p.M, p.dim, 23)
    g0 = torch.tensor(G0, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), "cuda")
    fc.cq_test_expire_waits(True)
    try:
        with pytest.raises(fc.CQError) as err:
            fc.fp2s_solve(cp, g0, gN, ws)
    finally:
        fc.cq_test_expire_waits(False)
    assert err.value.status == fc.CQ_ETIMEOUT
    fc.fp2s_solve(cp, g0, gN, ws)
    ref = OS.solve(p, G0)
    got = gN.cpu().numpy()
    assert max(float(np.linalg.norm(got[s] - ref[s]) / np.linalg.norm(ref[s])) for s in range(2)) <= 1e-4


def test_expired_wait_in_standalone_history(fc):
    ndof, n_lo, n_hi, beta, tau = 700, 1, 400, 0.6, 1.0 / 400
    G = ci.rng(31).standard_normal((n_hi, ndof))
    Gd = torch.tensor(G, device="cuda")
    H = torch.zeros(n_hi - n_lo, ndof, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, None, ndof, None, ndof,
                                           prec=fc.CQ_BF16X3), "cuda")
    fc.cq_test_expire_waits(True)
    try:
        fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, Gd, ndof, H, ndof, ws, prec=fc.CQ_BF16X3)
        torch.cuda.synchronize()
    finally:
        fc.cq_test_expire_waits(False)
    assert torch.isnan(H).any()
    fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, Gd, ndof, H, ndof, ws, prec=fc.CQ_BF16X3)
    torch.cuda.synchronize()
    got = H.cpu().numpy()
    d = OW.weights(1, beta, tau, n_hi)
    ref = OH.history_direct_all(d, G, n_lo, n_hi)
    # the BF16x3 bound: (3 * 2^-16 + K * 2^-24) * sum_i |d_i| |G^{n-i}| per element
    scale = np.stack([np.abs(d[n - 1:0:-1]) @ np.abs(G[1:n]) if n >= 2 else np.zeros(ndof)
                      for n in range(n_lo, n_hi)])
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= (3 * 2.0 ** -16 + n_hi * 2.0 ** -24) * scale + 1e-300)
