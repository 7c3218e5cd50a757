"""GPU test of cq_history_fast_noalloc, the fast-history entry point without a
workspace argument (``-m gpu``).

Some callers of this library cannot allocate device memory. Examples: a
plug-in that a host application hands nothing but its input and output
arrays, a program whose memory pool is fully reserved before its time loop,
or a loop that must not call cudaMalloc because that call can synchronise the
device and can fail at an arbitrary step. For them cq_history_fast_noalloc
keeps the history state in a fixed device array owned by the library.

The test drives the entry point through the C ABI for complete step sequences
in a row, in the three precisions it accepts (CQ_F64; CQ_F32, which lays out
padded FP32 rows and an FP32 table in the same array; CQ_DF64, double-float
rows and tables). Each later sequence is a
different problem, so it starts from whatever the previous one left in the
shared array, including a switch of precision between two problems. Every
step's h^n must agree with cq_history_fast (the workspace version) at the same
precision, within the tolerance of the other history tests:
|difference| <= 1e-12 (FP64, double-float) or 2e-5 (FP32) * sum_i |d_i| |G^{n-i}|. A request
that does not fit the array must be refused before any work is done. The file
is named so that pytest collects it last.
"""
import numpy as np
import pytest

import cq_inputs as ci
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


def _abs_scale(d, G, n):
    if n < 2:
        return np.zeros(G.shape[1])
    return np.abs(d[n - 1:0:-1]) @ np.abs(G[1:n])


def _run(fc, scheme, beta, np1, np2, ns, ndof, N, seed, prec=0):
    tol = 2e-5 if prec == fc.CQ_F32 else 1e-12
    tau = 1.0 / N
    G = ci.rng(seed).standard_normal((N + 1, ndof))
    Gd = torch.tensor(G, dtype=torch.float64, device="cuda")
    H_ws = torch.empty(ndof, dtype=torch.float64, device="cuda")
    H_na = torch.empty(ndof, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_fast(scheme, beta, tau, np1, np2, ns, ndof, 1, None, None, prec=prec), "cuda")
    d = OW.weights(scheme, beta, tau, N)
    for n in range(1, N + 1):
        fc.cq_history_fast(scheme, beta, tau, np1, np2, ns, ndof, n, Gd[n - 1], H_ws, ws, prec=prec)
        fc.cq_history_fast_noalloc(scheme, beta, tau, np1, np2, ns, ndof, n, Gd[n - 1], H_na, prec=prec)
        torch.cuda.synchronize()
        a = H_ws.cpu().numpy()
        b = H_na.cpu().numpy()
        assert np.all(np.abs(a - b) <= tol * _abs_scale(d, G, n) + 1e-300), n


def test_noalloc_matches_workspace_version_on_two_calls_in_a_row(fc):
    # first use: BDF2 fast form with the workload's sizes
    _run(fc, 2, 0.6, 16, 64, 17, 3001, 240, seed=31)
    # second use right after it: a different scheme and size on top of the leftovers
    _run(fc, 1, 0.3, 40, 0, 2, 777, 200, seed=32)


def test_noalloc_fp32_and_precision_switches(fc):
    # FP32 after the FP64 problems above, then FP64 on FP32 leftovers, then FP32 again
    _run(fc, 2, 0.45, 8, 24, 9, 2049, 180, seed=33, prec=fc.CQ_F32)
    _run(fc, 1, 0.55, 32, 0, 2, 1001, 150, seed=34, prec=fc.CQ_F64)
    _run(fc, 1, 0.7, 64, 0, 2, 4093, 160, seed=35, prec=fc.CQ_F32)


def test_noalloc_double_float_and_precision_switches(fc):
    # double-float on the leftovers of the problems above, FP32 on double-float leftovers,
    # then double-float again with the BE window
    _run(fc, 2, 0.6, 16, 64, 17, 2047, 200, seed=36, prec=fc.CQ_DF64)
    _run(fc, 2, 0.35, 8, 24, 9, 1500, 120, seed=37, prec=fc.CQ_F32)
    _run(fc, 1, 0.8, 48, 0, 2, 3001, 150, seed=38, prec=fc.CQ_DF64)


def test_noalloc_refuses_requests_that_do_not_fit(fc):
    H = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(fc.CQError) as e:
        fc.cq_history_fast_noalloc(2, 0.6, 1e-3, 16, 64, 17, 10_000_000, 1, None, H)
    assert e.value.status == fc.CQ_ENOMEM
