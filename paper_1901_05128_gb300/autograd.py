"""torch.autograd binding of the two-state solve.

``solve(G0, alpha, ...)`` returns G^N of the direct BE (Eq. 4.1) or SBD (Eq. 4.7)
scheme, or of the fast scheme (``fast = (np1, np2, ns)``), on the GPU (``fp2s_solve``). Its backward pass is the discrete adjoint of the
same scheme (``fp2s_vjp``): the transposed 2x2 steps run backwards in time with the CQ
convolution reversed in time, plus the beta-derivatives of the weights for the
gradient with respect to alpha_1, alpha_2 (d/dalpha_i = -d/dbeta_i, beta_i = 1 - alpha_i).
The backward pass recomputes the forward history inside the library call, so nothing
but G^0 and alpha is kept between forward and backward.

Both passes run on the device in FP64, in double-float (prec = CQ_DF64), or (prec =
CQ_BF16X3 / CQ_TF32X3, direct scheme) in the mixed-precision form: tensor-core histories on
FP32 levels, forward and adjoint alike.
Arguments are marshalled only.
"""
from __future__ import annotations

import torch

from . import fastcq as fc


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, G0, alpha, m, T, N, dim, M, scheme, prec, fast):
        a1, a2 = (float(v) for v in alpha.detach().cpu().tolist())
        if fast is None:
            p = fc.problem(a1, a2, m, T, N, dim, M, scheme, fc.CQ_DIRECT, prec=prec)
        else:
            p = fc.problem(a1, a2, m, T, N, dim, M, scheme, fc.CQ_FAST, *fast, prec=prec)
        G0c = G0.detach().contiguous()
        GN = torch.empty_like(G0c)
        ws = fc.workspace(fc.fp2s_solve(p, G0c, GN, None), G0c.device)
        fc.fp2s_solve(p, G0c, GN, ws)                   # on torch's current stream
        ctx.save_for_backward(G0c, alpha)
        ctx.p = p
        return GN

    @staticmethod
    def backward(ctx, dGN):
        G0, alpha = ctx.saved_tensors
        dG0 = torch.empty_like(G0)
        ws = fc.workspace(fc.fp2s_vjp(ctx.p, G0, dGN, dG0, None), G0.device)
        da = fc.fp2s_vjp(ctx.p, G0, dGN.contiguous(), dG0, ws)
        dalpha = torch.tensor(da, dtype=alpha.dtype, device=alpha.device)
        return dG0, dalpha, None, None, None, None, None, None, None, None


def solve(G0: torch.Tensor, alpha: torch.Tensor, *, m: float, T: float, N: int, dim: int, M: int,
          scheme: int = fc.CQ_BDF2, prec: int = fc.CQ_F64, fast=None) -> torch.Tensor:
    """G^N of the direct scheme (or, with fast = (np1, np2, ns), of the fast scheme) for G0
    (float64 CUDA tensor [2, M**dim]) and alpha = (alpha_1, alpha_2) (float64 tensor [2]);
    differentiable in both. prec: CQ_F64 or CQ_DF64; for the direct scheme also CQ_BF16X3 /
    CQ_TF32X3 for the mixed-precision form."""
    allowed = (fc.CQ_F64, fc.CQ_DF64) if fast is not None else (fc.CQ_F64, fc.CQ_DF64, fc.CQ_BF16X3, fc.CQ_TF32X3)
    if prec not in allowed:
        raise ValueError("prec must be one of %s for this form" % (allowed,))
    if fast is not None and len(fast) != 3:
        raise ValueError("fast must be (np1, np2, ns)")
    if G0.dtype != torch.float64 or not G0.is_cuda or tuple(G0.shape) != (2, M ** dim):
        raise ValueError("G0 must be a float64 CUDA tensor of shape (2, M**dim)")
    if alpha.numel() != 2:
        raise ValueError("alpha must hold (alpha_1, alpha_2)")
    return _Solve.apply(G0, alpha, m, T, N, dim, M, scheme, prec, None if fast is None else tuple(fast))
