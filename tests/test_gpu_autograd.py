"""Backward pass of the direct solve for an arbitrary upstream gradient (fp2s_vjp) and
its torch.autograd binding (``-m gpu``).

- fp2s_vjp with dL/dG^N = h^dim (G^N - Gt) is the misfit gradient, so it must equal
  fp2s_gradient (same adjoint sweep, same arithmetic): 1e-13 relative.
- The solve is linear in G0, so a central difference of L = <W, G^N> along a direction
  is exact up to rounding: <dL/dG0, V> agrees to 1e-10 relative.
- dL/dalpha against central differences of the GPU forward solve (step 1e-5, FP64;
  accurate to ~1e-9 relative): 1e-6 relative.
- torch.autograd.gradcheck on a tiny problem (every G0 entry and both alphas).
- The mixed-precision binding (prec = CQ_BF16X3) against the FP64 one, within the mixed
  gradient's bars; dL/dalpha relative to max(|dL/dalpha|, |L|), since a random W can make
  dL/dalpha small against the terms it sums.
"""
import numpy as np
import pytest

import cq_inputs as ci

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_05128_gb300 as pkg
    pkg.build()
    from paper_1901_05128_gb300 import autograd as ag
    return pkg.load(), ag


CASES = [ci.Problem(0.3, 0.7, 0.4, 1.0, 40, 1, 15, ci.BE, ci.DIRECT),
         ci.Problem(0.4, 0.6, 0.4, 1.0, 50, 1, 21, ci.BDF2, ci.DIRECT),
         ci.Problem(0.25, 0.8, 0.6, 1.0, 29, 2, 9, ci.BDF2, ci.DIRECT)]


def _solve(fc, p, G0, a1=None, a2=None):
    cp = fc.problem(p.alpha1 if a1 is None else a1, p.alpha2 if a2 is None else a2, p.m, p.T, p.N, p.dim, p.M,
                    p.scheme, ci.DIRECT)
    gN = torch.empty_like(G0)
    ws = fc.workspace(fc.fp2s_solve(cp, G0, gN, None), "cuda")
    fc.fp2s_solve(cp, G0, gN, ws)
    return gN


@pytest.mark.parametrize("p", CASES, ids=["be_1d", "bdf2_1d", "bdf2_2d"])
def test_vjp_equals_misfit_gradient(pkg, p):
    fc, _ = pkg
    cp = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, ci.DIRECT)
    G0 = torch.tensor(ci.g0_uniform(p.M, p.dim, 5), dtype=torch.float64, device="cuda")
    Gt = torch.tensor(ci.g0_uniform(p.M, p.dim, 6), dtype=torch.float64, device="cuda") * 0.1
    dg = torch.empty_like(G0)
    ws = fc.workspace(fc.fp2s_gradient(cp, G0, Gt, dg, None), "cuda")
    assert fc.fp2s_vjp(cp, G0, Gt, dg, None) == ws.numel()
    J, da = fc.fp2s_gradient(cp, G0, Gt, dg, ws)
    GN = _solve(fc, p, G0)
    h = 1.0 / (p.M + 1)
    up = (h ** p.dim) * (GN - Gt)
    dv = torch.empty_like(G0)
    dav = fc.fp2s_vjp(cp, G0, up, dv, ws)
    assert np.allclose(dav, da, rtol=1e-13, atol=0)
    assert torch.max(torch.abs(dv - dg)) <= 1e-13 * torch.max(torch.abs(dg))


@pytest.mark.parametrize("p", CASES, ids=["be_1d", "bdf2_1d", "bdf2_2d"])
def test_autograd_against_differences(pkg, p):
    fc, ag = pkg
    rng = ci.rng(77)
    G0 = torch.tensor(ci.g0_uniform(p.M, p.dim, 8), dtype=torch.float64, device="cuda", requires_grad=True)
    alpha = torch.tensor([p.alpha1, p.alpha2], dtype=torch.float64, device="cuda", requires_grad=True)
    W = torch.tensor(rng.standard_normal((2, p.M ** p.dim)), dtype=torch.float64, device="cuda")
    GN = ag.solve(G0, alpha, m=p.m, T=p.T, N=p.N, dim=p.dim, M=p.M, scheme=p.scheme)
    L = torch.sum(W * GN)
    L.backward()
    # G0 direction: exact for a linear map
    V = torch.tensor(rng.standard_normal((2, p.M ** p.dim)), dtype=torch.float64, device="cuda")
    with torch.no_grad():
        eps = 1e-3
        Lp = torch.sum(W * _solve(fc, p, G0 + eps * V)).item()
        Lm = torch.sum(W * _solve(fc, p, G0 - eps * V)).item()
        fd = (Lp - Lm) / (2 * eps)
        an = torch.sum(G0.grad * V).item()
        assert abs(fd - an) <= 1e-10 * max(abs(fd), 1e-300)
        for i in range(2):
            h = 1e-5
            a_p = [p.alpha1, p.alpha2]
            a_m = [p.alpha1, p.alpha2]
            a_p[i] += h
            a_m[i] -= h
            fdi = (torch.sum(W * _solve(fc, p, G0, *a_p)).item() - torch.sum(W * _solve(fc, p, G0, *a_m)).item()) / (2 * h)
            assert abs(fdi - alpha.grad[i].item()) <= 1e-6 * abs(fdi), (i, fdi, alpha.grad[i].item())


def test_gradcheck_tiny(pkg):
    fc, ag = pkg
    G0 = torch.tensor(ci.g0_uniform(5, 1, 3), dtype=torch.float64, device="cuda", requires_grad=True)
    alpha = torch.tensor([0.35, 0.65], dtype=torch.float64, device="cuda", requires_grad=True)

    def f(g, a):
        return ag.solve(g, a, m=0.3, T=1.0, N=12, dim=1, M=5, scheme=fc.CQ_BDF2)

    assert torch.autograd.gradcheck(f, (G0, alpha), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_gradcheck_tiny_fast_form(pkg):
    """The fast scheme through the binding (fast = (np1, np2, ns)): torch's gradcheck against
    central differences in G0 and alpha (the quadrature tables rebuilt at every perturbed alpha)."""
    fc, ag = pkg
    G0 = torch.tensor(ci.g0_uniform(5, 1, 4), dtype=torch.float64, device="cuda", requires_grad=True)
    alpha = torch.tensor([0.35, 0.65], dtype=torch.float64, device="cuda", requires_grad=True)

    def f(g, a):
        return ag.solve(g, a, m=0.3, T=1.0, N=24, dim=1, M=5, scheme=fc.CQ_BDF2, fast=(4, 8, 5))

    assert torch.autograd.gradcheck(f, (G0, alpha), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_autograd_rejects_bad_input(pkg):
    fc, ag = pkg
    a = torch.tensor([0.3, 0.6], dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ag.solve(torch.zeros(2, 7, dtype=torch.float32, device="cuda"), a, m=0.3, T=1.0, N=4, dim=1, M=7)
    with pytest.raises(ValueError):
        ag.solve(torch.zeros(2, 6, dtype=torch.float64, device="cuda"), a, m=0.3, T=1.0, N=4, dim=1, M=7)
    with pytest.raises(ValueError):               # no mixed-precision fast-form gradient
        ag.solve(torch.zeros(2, 7, dtype=torch.float64, device="cuda"), a, m=0.3, T=1.0, N=4, dim=1, M=7,
                 fast=(4, 8, 5), prec=fc.CQ_BF16X3)


@pytest.mark.parametrize("p", CASES, ids=["be_1d", "bdf2_1d", "bdf2_2d"])
def test_autograd_mixed_precision_against_fp64(pkg, p):
    """prec = CQ_BF16X3: forward and backward through the mixed-precision form; the
    gradients match the FP64 binding's within the mixed gradient's bars (test_gpu_mixed_gradient)."""
    fc, ag = pkg
    rng = ci.rng(78)
    W = torch.tensor(rng.standard_normal((2, p.M ** p.dim)), dtype=torch.float64, device="cuda")
    grads, Ls = [], []
    for prec in (fc.CQ_F64, fc.CQ_BF16X3):
        G0 = torch.tensor(ci.g0_uniform(p.M, p.dim, 8), dtype=torch.float64, device="cuda", requires_grad=True)
        alpha = torch.tensor([p.alpha1, p.alpha2], dtype=torch.float64, device="cuda", requires_grad=True)
        GN = ag.solve(G0, alpha, m=p.m, T=p.T, N=p.N, dim=p.dim, M=p.M, scheme=p.scheme, prec=prec)
        L = torch.sum(W * GN)
        L.backward()
        Ls.append(abs(L.item()))
        grads.append((GN.detach(), G0.grad, alpha.grad))
    (g64, dg64, da64), (gmx, dgmx, damx) = grads
    assert torch.linalg.norm(gmx - g64) <= 1e-4 * torch.linalg.norm(g64)
    assert torch.linalg.norm(dgmx - dg64) <= 2e-4 * torch.linalg.norm(dg64)
    assert torch.all(torch.abs(damx - da64) <= 5e-4 * torch.clamp(torch.abs(da64), min=Ls[0]))
    with pytest.raises(ValueError):
        ag.solve(torch.zeros(2, p.M ** p.dim, dtype=torch.float64, device="cuda"), torch.tensor([0.3, 0.6]), m=p.m,
                 T=p.T, N=p.N, dim=p.dim, M=p.M, prec=fc.CQ_F32)
