"""Empty inputs of the history entry points (eq. 4.1 / 4.7 sums over no step or no DOF):
an empty step range or zero DOFs returns CQ_OK, launches nothing and leaves the output
untouched, in every precision."""
import numpy as np
import pytest
import torch

from paper_1901_05128_gb300 import fastcq as fc

pytestmark = pytest.mark.gpu

PRECS = [fc.CQ_F64, fc.CQ_BF16X3, fc.CQ_TF32X3]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("ndof,n_lo,n_hi", [(100, 7, 7), (0, 1, 50), (0, 3, 3)])
def test_history_direct_empty(prec, ndof, n_lo, n_hi):
    ld = max(ndof, 4)
    G = torch.randn(max(n_hi, 1), ld, dtype=torch.float64, device="cuda")
    H = torch.full((2, ld), float("nan"), dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_direct(1, 0.4, 1e-2, ndof, n_lo, n_hi, None, ld, None, ld, prec=prec))
    torch.cuda.synchronize()
    k0 = fc.cq_launch_count()
    fc.cq_history_direct(1, 0.4, 1e-2, ndof, n_lo, n_hi, G, ld, H, ld, ws, prec=prec)
    torch.cuda.synchronize()
    assert fc.cq_launch_count() == k0
    assert torch.isnan(H).all()


@pytest.mark.parametrize("prec", [fc.CQ_F64, fc.CQ_F32])
@pytest.mark.parametrize("scheme,np1,np2,ns", [(1, 16, 0, 2), (2, 8, 8, 5)])
def test_history_fast_zero_dofs(prec, scheme, np1, np2, ns):
    H = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    G = torch.zeros(4, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_fast(scheme, 0.6, 1e-2, np1, np2, ns, 0, 1, None, None, prec=prec))
    k0 = fc.cq_launch_count()
    for n in range(1, 6):
        fc.cq_history_fast(scheme, 0.6, 1e-2, np1, np2, ns, 0, n, G, H, ws, prec=prec)
    torch.cuda.synchronize()
    assert fc.cq_launch_count() == k0
    assert np.isnan(H.cpu().numpy()).all()
