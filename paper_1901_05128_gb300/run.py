"""Command-line runner: solve one named synthetic workload on the GPU.

    python -m paper_1901_05128_gb300.run --workload bdf2_2d_m255 --form fast --repeat 2
    python -m paper_1901_05128_gb300.run --workload grad_2d_m255 --gradient --prec bf16x3 --scale-exp 0
    python -m paper_1901_05128_gb300.run --fast-history --prec df64 --ndof 1048576 --repeat 8
    python -m paper_1901_05128_gb300.run --batch 16 --prec df64 --repeat 2

Prints one line per solve (or gradient) with its wall time and the library status.
Useful for profiling a single configuration (e.g. under ncu).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="bdf2_2d_m255")
    ap.add_argument("--form", choices=["fast", "direct"], default=None)
    ap.add_argument("--scheme", choices=["be", "bdf2"], default=None)
    ap.add_argument("--N", type=int, default=None, help="override the number of steps")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--scale-exp", type=int, default=-1000, help="G0 is multiplied by 2**scale_exp")
    ap.add_argument("--prec", choices=["f64", "f32", "bf16x3", "tf32x3", "df64"], default="f64")
    ap.add_argument("--history", action="store_true",
                    help="run cq_history_direct alone on synthetic N(0,1) levels (--ndof, --n-lo, --n-hi)")
    ap.add_argument("--gradient", action="store_true",
                    help="run fp2s_gradient of the workload (direct form, or --form fast in FP64) against a "
                         "target made with alpha + (0.05, -0.05)")
    ap.add_argument("--fast-history", action="store_true",
                    help="run cq_history_fast one step at a time on synthetic N(0,1) levels (--ndof DOFs; "
                         "BDF2 sizes np1 = 16, np2 = 64, Ns = 17; --repeat timed steps past the exact window)")
    ap.add_argument("--batch", type=int, default=0, metavar="K",
                    help="solve the first K instances of the seeded uneven-instance batch workload in one "
                         "persistent launch (fp2s_batch_plan, autotuned, then fp2s_solve_batched)")
    ap.add_argument("--ndof", type=int, default=65536)
    ap.add_argument("--n-lo", type=int, default=1)
    ap.add_argument("--n-hi", type=int, default=2049)
    a = ap.parse_args(argv)

    import torch

    import cq_inputs as ci
    from . import build, load

    build()
    fc = load()
    if a.history:
        return run_history(fc, torch, a)
    if a.fast_history:
        return run_fast_history(fc, torch, a)
    if a.batch:
        return run_batch(fc, torch, a)
    p, G0 = ci.workload(a.workload)
    if a.form:
        p = p.replace(form=ci.FAST if a.form == "fast" else ci.DIRECT)
    if a.scheme:
        p = p.replace(scheme=ci.BE if a.scheme == "be" else ci.BDF2)
    if a.N:
        p = p.replace(N=a.N, T=p.T * a.N / p.N)
    prec = {"f64": fc.CQ_F64, "f32": fc.CQ_F32, "bf16x3": fc.CQ_BF16X3, "tf32x3": fc.CQ_TF32X3,
            "df64": fc.CQ_DF64}[a.prec]
    cp = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                    prec=prec)
    g0 = torch.tensor(G0 * 2.0 ** a.scale_exp, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    if a.gradient:
        return run_gradient(fc, torch, a, p, cp, g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None))
    fc.cq_timing_enable(True)
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        st = fc.fp2s_solve(cp, g0, gN, ws, check=False)
        torch.cuda.synchronize()
        print("solve %d: %.3f s (time-stepping %.3f ms) status=%s"
              % (r, time.perf_counter() - t, fc.cq_timing_last(), fc.strerror(st)))


def run_gradient(fc, torch, a, p, cp, g0):
    """Gradient of 1/2 ||G^N - G_target||^2 (the run's form and precision; the fast form in FP64
    only); the target is the FP64 direct solve with alpha + (0.05, -0.05). Prints the time per
    gradient."""
    import cq_inputs as ci
    ct = fc.problem(p.alpha1 + 0.05, p.alpha2 - 0.05, p.m, p.T, p.N, p.dim, p.M, p.scheme, ci.DIRECT)
    gt = torch.empty_like(g0)
    fc.fp2s_solve(ct, g0, gt, fc.workspace(fc.fp2s_solve(ct, g0, gt, None)))
    dg = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_gradient(cp, g0, gt, dg, None))
    fc.cq_timing_enable(True)
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        J, da = fc.fp2s_gradient(cp, g0, gt, dg, ws)
        torch.cuda.synchronize()
        print("gradient %d: %.3f ms (kernels %.3f ms, contractions %.3f ms) J=%.6e dJ/dalpha=(%.6e, %.6e)"
              % (r, (time.perf_counter() - t) * 1e3, fc.cq_timing_last(), fc.cq_timing_part(1), J, da[0], da[1]))


def run_history(fc, torch, a):
    """Direct history of synthetic levels: prints call and main-kernel times."""
    import cq_inputs as ci
    prec = {"f64": fc.CQ_F64, "bf16x3": fc.CQ_BF16X3, "tf32x3": fc.CQ_TF32X3}.get(a.prec)
    if prec is None:
        raise SystemExit("--history supports --prec f64, bf16x3 or tf32x3")
    ndof, n_lo, n_hi = a.ndof, a.n_lo, a.n_hi
    beta, tau = 0.8, 1.0 / max(n_hi - 1, 1)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(ci.SEED_BASE + 7)
    G = torch.randn(n_hi, ndof, dtype=torch.float64, device="cuda", generator=gen)
    H = torch.empty(n_hi - n_lo, ndof, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, None, ndof, None, ndof, prec=prec))
    fc.cq_timing_enable(True)
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        fc.cq_history_direct(1, beta, tau, ndof, n_lo, n_hi, G, ndof, H, ndof, ws, prec=prec)
        torch.cuda.synchronize()
        k = fc.cq_timing_last() if prec in (fc.CQ_BF16X3, fc.CQ_TF32X3) else float("nan")
        print("history %d: %.3f ms (main kernel %.3f ms)" % (r, (time.perf_counter() - t) * 1e3, k))


def run_fast_history(fc, torch, a):
    """Per-step fast history (SBD sizes np1 = 16, np2 = 64, Ns = 17, beta = 0.6, tau = 1/4096) over
    --ndof DOFs: Ns + 8 untimed steps, then --repeat steps; prints each step's kernel time."""
    import cq_inputs as ci
    prec = {"f64": fc.CQ_F64, "f32": fc.CQ_F32, "df64": fc.CQ_DF64}.get(a.prec)
    if prec is None:
        raise SystemExit("--fast-history supports --prec f64, f32 or df64")
    np1, np2, ns, beta, tau, ndof = 16, 64, 17, 0.6, 1.0 / 4096, a.ndof
    gen = torch.Generator(device="cuda")
    gen.manual_seed(ci.SEED_BASE + 8)
    G = torch.randn(2, ndof, dtype=torch.float64, device="cuda", generator=gen)
    H = torch.empty(ndof, dtype=torch.float64, device="cuda")
    ws = fc.workspace(fc.cq_history_fast(2, beta, tau, np1, np2, ns, ndof, 1, None, None, prec=prec))
    fc.cq_timing_enable(True)
    n = 1
    for _ in range(ns + 8):
        fc.cq_history_fast(2, beta, tau, np1, np2, ns, ndof, n, G[n % 2], H, ws, prec=prec)
        n += 1
    torch.cuda.synchronize()
    for r in range(a.repeat):
        fc.cq_history_fast(2, beta, tau, np1, np2, ns, ndof, n, G[n % 2], H, ws, prec=prec)
        print("fast history step %d: kernel %.3f ms" % (n, fc.cq_timing_last()))
        n += 1


def run_batch(fc, torch, a):
    """The first --batch instances of the seeded batch workload in one persistent launch, in the
    run's precision (f64 or df64), each shortened to at most --N steps if given; prints the time per
    batch and the batch status."""
    import numpy as np
    import cq_inputs as ci
    prec = {"f64": fc.CQ_F64, "df64": fc.CQ_DF64}.get(a.prec)
    if prec is None:
        raise SystemExit("--batch supports --prec f64 or df64")
    probs, fields, _ = ci.batch_workload()
    probs, fields = probs[:a.batch], fields[:a.batch]
    if a.N:                                  # shorten every instance to at most --N steps (same tau)
        probs = [p.replace(N=min(p.N, a.N), T=p.T * min(p.N, a.N) / p.N) for p in probs]
    cps = [fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                      prec=prec, flags=fc.FP2S_ASYNC) for p in probs]
    ws = fc.workspace(fc.fp2s_batch_plan(cps))
    plan = fc.fp2s_batch_plan(cps, ws, tune=prec == fc.CQ_F64)
    print("plan: %d warps per block, %d CTAs per SM (0: all that fit), node-loop width %d; %d candidates "
          "timed (%d solve launches while tuning)" % (plan.warps_per_block, plan.ctas_per_sm, plan.node_unroll,
                                                     plan.tuned_candidates, 4 * plan.tuned_candidates))
    g0 = torch.tensor(np.concatenate([f.reshape(-1) for f in fields]) * 2.0 ** a.scale_exp,
                      dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    fc.cq_timing_enable(True)
    units = sum(2 * p.M ** p.dim * p.N for p in probs)
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        fc.fp2s_solve_batched(plan, g0, gN, ws)
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        print("batch %d: %d instances, %.3f ms (kernels %.3f ms), %.3e DOF-steps/s, status=%s"
              % (r, len(probs), el * 1e3, fc.cq_timing_last(), units / el,
                 fc.strerror(fc.fp2s_batch_status(plan, ws))))


if __name__ == "__main__":
    main()
