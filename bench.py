#!/usr/bin/env python
"""Benchmark of the CQ history hot path on GB300.

Workload (one "step" = one whole fp2s_solve: CQ weights, Gauss-Jacobi fast
coefficients, forward sine transform, all N time steps with the history sums
and the per-mode 2x2 solves, inverse sine transform):
  2D unit square, 255 x 255 interior finite-difference points (2 x 65025 DOF),
  T = 1, N = 4096, BDF2 (SBD) scheme, alpha = (0.4, 0.6), m = 0.49, fast form
  with N_p1 = 16, N_p2 = 64, N_s = 17, FP64; G0 = seeded U[0,1) on an 8x8
  checkerboard, times 2^-1000 (the problem is linear; the factor keeps the mode
  that grows like e^(1096 t) finite without changing the arithmetic).
The same workload is also timed in the direct form ("direct" sub-object).

value = DOF x N / (device time of one step), summed over ranks (weak scaling:
every rank solves its own instance). L2 is flushed (256 MiB write) before
every timed step, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# The oracle legs run on one host thread and report cores = 1: their per-step numpy arithmetic is
# element-wise, and the vector-matrix products of the direct history must not fan out to BLAS
# threads either (set before numpy is first imported).
for _var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_var] = "1"

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CQ history DOF·steps/s (fast vs direct, FP64 vs mixed) at stated error; grad steps/s"
UNIT = "DOF·steps/s"
WORKLOAD = "bdf2_2d_m255"
SCALE = 2.0 ** -1000
FP64_PEAK_NOMINAL = 1.25e12       # FP64 FLOP/s of GB300 (2 DFMA / clock / SM x 152 SMs x ~2.07 GHz)
FP64_PEAK_PROBE = 1.199e12        # own DFMA-chain probe on this machine's GB300 (independent FMA chains)
FP32_PEAK_PROBE = 73.2e12         # own FFMA-chain probe, same method
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def workload_config(p):
    return {
        "workload": "%s: 2D %dx%d FD grid (%d DOF), T=%g, N=%d, BDF2, alpha=(%g,%g), m=%g, fast np1=%d np2=%d Ns=%d, "
                    "G0 = U[0,1) checkerboard x 2^-1000" % (WORKLOAD, p.M, p.M, p.ndof, p.T, p.N, p.alpha1,
                                                           p.alpha2, p.m, p.np1, p.np2, p.ns),
        "dof": p.ndof, "N": p.N, "scheme": "BDF2", "form": "fast", "precision": "FP64",
        "l2": "flushed before every timed step (256 MiB write), outside the timed events",
    }


# ----------------------------------------------------------------------------- oracle (CPU) legs
def oracle_sample(p, G0, n_modes, seed):
    """Time the oracle's plain per-mode scheme on a seeded sample of sine modes."""
    import numpy as np
    from oracle import scheme as OS
    from oracle import spatial as OSP
    import cq_inputs as ci

    nm = p.M ** p.dim
    lowest = [0, 1, p.M, p.M + 1] if p.dim == 2 else [0, 1]
    sample = np.unique(np.concatenate([lowest, ci.sample_indices(nm, n_modes, seed)]))
    lam = OSP.mode_eigenvalues(p.M, p.dim)[sample]
    g0 = OSP.to_modal(G0, p.M, p.dim)[:, sample]
    t = time.perf_counter()
    g = OS.solve_modal(p, lam, g0)
    dt = time.perf_counter() - t
    return sample, g[p.N], dt


def cpu_cores_used():
    return 1        # the oracle's time loop is numpy element-wise work on one thread


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + SMI_FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ----------------------------------------------------------------------------- precision forms
PREC_WORKLOAD = "prec_2d_m511"
PREC_COLS = 16


def precision_leg(fc, torch, dev, K, W, flush):
    """Tensor-core (BF16x3) direct history over the full 2D 511x511, N = 8192 contraction,
    and the FP32 fast solve of the same grid. Returns timings plus the data the CPU leg
    needs to state the error against the oracle."""
    import cq_inputs as ci
    p, G0 = ci.workload(PREC_WORKLOAD)
    n_hi, ndof = p.N + 1, p.ndof
    beta, tau = 1.0 - p.alpha1, p.T / p.N
    out = {"problem": p}
    gen = torch.Generator(device=dev)
    gen.manual_seed(ci.SEED_BASE + 3)
    G = torch.randn(n_hi, ndof, dtype=torch.float64, device=dev, generator=gen)   # synthetic levels
    H = torch.empty(n_hi - 1, ndof, dtype=torch.float64, device=dev)
    ws = fc.workspace(fc.cq_history_direct(ci.BE, beta, tau, ndof, 1, n_hi, None, ndof, None, ndof,
                                           prec=fc.CQ_BF16X3), dev)
    for _ in range(W):
        fc.cq_history_direct(ci.BE, beta, tau, ndof, 1, n_hi, G, ndof, H, ndof, ws, prec=fc.CQ_BF16X3)
    torch.cuda.synchronize()
    l0 = fc.cq_launch_count()
    calls, gemms = [], []
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fc.cq_history_direct(ci.BE, beta, tau, ndof, 1, n_hi, G, ndof, H, ndof, ws, prec=fc.CQ_BF16X3)
        e1.record()
        e1.synchronize()
        calls.append(e0.elapsed_time(e1))
        gemms.append(fc.cq_timing_last())
    out["tc_launches"] = fc.cq_launch_count() - l0
    cols = ci.sample_indices(ndof, PREC_COLS, ci.SEED_BASE + 31)
    ci_t = torch.tensor(cols, device=dev)
    out["tc_cols"] = cols
    out["tc_G"] = G[:, ci_t].cpu().numpy()
    out["tc_H"] = H[:, ci_t].cpu().numpy()
    out["tc_call_ms"], out["tc_gemm_ms"] = calls, gemms
    out["tc_beta"], out["tc_tau"], out["tc_nhi"] = beta, tau, n_hi
    # the same contraction in the TF32x3 form
    del ws
    torch.cuda.empty_cache()
    ws = fc.workspace(fc.cq_history_direct(ci.BE, beta, tau, ndof, 1, n_hi, None, ndof, None, ndof,
                                           prec=fc.CQ_TF32X3), dev)
    for _ in range(W):
        fc.cq_history_direct(ci.BE, beta, tau, ndof, 1, n_hi, G, ndof, H, ndof, ws, prec=fc.CQ_TF32X3)
    torch.cuda.synchronize()
    tcalls, tgemms = [], []
    for _ in range(max(3, K // 3)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fc.cq_history_direct(ci.BE, beta, tau, ndof, 1, n_hi, G, ndof, H, ndof, ws, prec=fc.CQ_TF32X3)
        e1.record()
        e1.synchronize()
        tcalls.append(e0.elapsed_time(e1))
        tgemms.append(fc.cq_timing_last())
    out["tf32_H"] = H[:, ci_t].cpu().numpy()
    out["tf32_call_ms"], out["tf32_gemm_ms"] = tcalls, tgemms
    del G, H, ws
    torch.cuda.empty_cache()
    # FP32 fast solve of the same grid
    q = p.replace(form=ci.FAST)
    cp = fc.problem(q.alpha1, q.alpha2, q.m, q.T, q.N, q.dim, q.M, q.scheme, q.form, q.np1, q.np2, q.ns,
                    prec=fc.CQ_F32, flags=fc.FP2S_ASYNC)
    g0 = torch.tensor(G0, dtype=torch.float64, device=dev)
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), dev)
    for _ in range(W):
        fc.fp2s_solve(cp, g0, gN, ws)
    torch.cuda.synchronize()
    steps, kern = [], []
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fc.fp2s_solve(cp, g0, gN, ws)
        e1.record()
        e1.synchronize()
        steps.append(e0.elapsed_time(e1))
        kern.append(fc.cq_timing_last())
    out["f32_status"] = fc.strerror(fc.fp2s_status(cp, ws))
    out["f32_ms"], out["f32_kernel_ms"] = steps, kern
    out["f32_gN"] = gN.cpu().numpy()
    out["f32_problem"], out["G0"] = q, G0
    del ws, g0, gN
    torch.cuda.empty_cache()
    out["mixed"] = mixed_direct_leg(fc, torch, dev, p, G0, K, W, flush)
    return out


MIXED_ALPHAS = ((0.2, 0.8), (0.8, 0.2), (0.2, 0.2), (0.8, 0.8))


def mixed_direct_leg(fc, torch, dev, p, G0, K, W, flush):
    """Mixed-precision direct solve (tensor-core BF16x3 history, FP32 in-block sums and
    steps) of the 2D 511x511, N = 8192 grid for BE and BDF2 and every (alpha1, alpha2) in
    {0.2, 0.8}^2, and the BE (0.2, 0.8) case with the TF32x3 contraction. The first case
    (BE, alpha = (0.2, 0.8), BF16x3) is timed K times; the others once."""
    import cq_inputs as ci
    runs = []
    g0 = torch.tensor(G0, dtype=torch.float64, device=dev)
    gN = torch.empty_like(g0)
    ws = None
    cases = [(scheme, al, fc.CQ_BF16X3) for scheme in (ci.BE, ci.BDF2) for al in MIXED_ALPHAS]
    cases.append((ci.BE, MIXED_ALPHAS[0], fc.CQ_TF32X3))
    for scheme, al, prec in cases:
        q = p.replace(form=ci.DIRECT, scheme=scheme, alpha1=al[0], alpha2=al[1])
        cp = fc.problem(q.alpha1, q.alpha2, q.m, q.T, q.N, q.dim, q.M, q.scheme, q.form, 0, 0, 0,
                        prec=prec, flags=fc.FP2S_ASYNC)
        if prec == fc.CQ_TF32X3:          # twice the level bytes: a larger workspace
            ws = None
            torch.cuda.empty_cache()
        if ws is None:
            ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), dev)
        main = not runs
        for _ in range(W if main else 1):
            fc.fp2s_solve(cp, g0, gN, ws)
        torch.cuda.synchronize()
        l0 = fc.cq_launch_count()
        ms, tc_ms = [], []
        for _ in range(K if main else 1):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fc.fp2s_solve(cp, g0, gN, ws)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            tc_ms.append(fc.cq_timing_part(1))
        runs.append({"problem": q, "prec": "tf32x3" if prec == fc.CQ_TF32X3 else "bf16x3", "ms": ms,
                     "tc_ms": tc_ms, "status": fc.strerror(fc.fp2s_status(cp, ws)),
                     "launches": (fc.cq_launch_count() - l0) / len(ms), "gN": gN.cpu().numpy()})
    # the main case's levels at earlier steps n (same tau: N = n, T = n tau), for its per-step error
    q0 = runs[0]["problem"]
    partial = {}
    for n in (q0.N // 8, q0.N // 4, q0.N // 2, 3 * q0.N // 4):
        qn = q0.replace(N=n, T=q0.T * n / q0.N)
        cpn = fc.problem(qn.alpha1, qn.alpha2, qn.m, qn.T, qn.N, qn.dim, qn.M, qn.scheme, qn.form, 0, 0, 0,
                         prec=fc.CQ_BF16X3)
        fc.fp2s_solve(cpn, g0, gN, ws)
        partial[n] = gN.cpu().numpy()
    runs[0]["partial"] = partial
    del ws, g0, gN
    torch.cuda.empty_cache()
    return runs


def precision_report(leg, cpu_modes):
    """Oracle comparison and CPU baseline of the precision forms (CPU leg)."""
    import numpy as np
    import cq_inputs as ci
    from oracle import history as OH
    from oracle import spatial as OSP
    from oracle import weights as OW
    p = leg["problem"]
    n_hi, ndof = leg["tc_nhi"], p.ndof
    rows = n_hi - 1
    # tensor-core contraction: the oracle recomputes PREC_COLS whole DOF columns
    d = OW.weights(ci.BE, leg["tc_beta"], leg["tc_tau"], n_hi)
    t = time.perf_counter()
    ref = OH.history_direct_all(d, leg["tc_G"], 1, n_hi)
    t_orc = time.perf_counter() - t
    scale = np.stack([np.abs(d[n - 1:0:-1]) @ np.abs(leg["tc_G"][1:n]) if n >= 2 else np.zeros(PREC_COLS)
                      for n in range(1, n_hi)])
    tc_err = float(np.max(np.abs(leg["tc_H"] - ref) / (scale + 1e-300)))
    gemm_ms = statistics.mean(leg["tc_gemm_ms"])
    call_ms = statistics.mean(leg["tc_call_ms"])
    useful = 3 * 2.0 * ndof * (rows * (rows - 1) / 2.0)
    peaks = _measured_peaks()
    bf16_peak = peaks.get("bf16_tflops", 1948.7)
    tc = {
        "workload": "%s: 2D %dx%d (%d DOF), levels 1..%d, BE weights beta=%g, tau=1/%d, synthetic N(0,1) levels"
                    % (PREC_WORKLOAD, p.M, p.M, ndof, n_hi - 1, leg["tc_beta"], p.N),
        "precision": "BF16x3 (hi*hi + hi*lo + lo*hi), FP32 accumulation, FP64 output",
        "value": ndof * rows / (call_ms * 1e-3), "unit": UNIT, "ms_per_call": call_ms,
        "gemm": {"value": ndof * rows / (gemm_ms * 1e-3), "ms": gemm_ms},
        "roofline": {"kernel": "k_history_tc<double, BF16X3>", "bound": "tensor", "unit": "TFLOP/s",
                     "achieved": useful / (gemm_ms * 1e-3) / 1e12, "peak": bf16_peak,
                     "frac": useful / (gemm_ms * 1e-3) / 1e12 / bf16_peak,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst; kernel timed alone)",
                     "algorithmic_flops_per_launch": useful,
                     "flops_definition": "3 products x 2 x ndof x sum_n (n-1) (strictly lower-triangular Toeplitz)"},
        "error_vs_oracle": {"max_abs_err_over_sum_abs_terms": tc_err, "bound": 3 * 2.0 ** -16 + rows * 2.0 ** -24,
                            "sample": "%d whole DOF columns x %d steps" % (PREC_COLS, rows)},
        "gpu_launches_per_call": leg["tc_launches"] / max(1, len(leg["tc_gemm_ms"])),
        "cpu_baseline": {"value": PREC_COLS * rows / t_orc, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "oracle direct history of %d DOF columns x %d steps (%.1f s)"
                                   % (PREC_COLS, rows, t_orc)},
    }
    tf_gemm = statistics.mean(leg["tf32_gemm_ms"])
    tf32_peak = bf16_peak * 1.1 / 2.25            # nominal TF32 : BF16 dense ratio
    tf_err = float(np.max(np.abs(leg["tf32_H"] - ref) / (scale + 1e-300)))
    tf32 = {
        "workload": tc["workload"],
        "precision": "TF32x3 (hi*hi + hi*lo + lo*hi, 11-bit parts), FP32 accumulation per 128-level chunk, "
                     "FP64 output",
        "value": ndof * rows / (statistics.mean(leg["tf32_call_ms"]) * 1e-3), "unit": UNIT,
        "ms_per_call": statistics.mean(leg["tf32_call_ms"]),
        "roofline": {"kernel": "k_history_tc<double, TF32X3>", "bound": "tensor", "unit": "TFLOP/s",
                     "achieved": useful / (tf_gemm * 1e-3) / 1e12, "peak": tf32_peak,
                     "frac": useful / (tf_gemm * 1e-3) / 1e12 / tf32_peak,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops x nominal TF32/BF16 ratio 1.1/2.25",
                     "kernel_ms": tf_gemm},
        "error_vs_oracle": {"max_abs_err_over_sum_abs_terms": tf_err,
                            "sample": "%d whole DOF columns x %d steps" % (PREC_COLS, rows)},
    }
    # FP32 fast solve: oracle FP64 fast scheme on sampled modes
    from oracle import scheme as OS
    q, G0 = leg["f32_problem"], leg["G0"]
    nm = q.M ** q.dim
    sample = np.unique(np.concatenate([[0, 1, q.M, q.M + 1], ci.sample_indices(nm, cpu_modes, ci.SEED_BASE + 32)]))
    lam = OSP.mode_eigenvalues(q.M, q.dim)[sample]
    g0 = OSP.to_modal(G0, q.M, q.dim)[:, sample]
    t = time.perf_counter()
    refm = OS.solve_modal(q, lam, g0)[q.N]
    t_f = time.perf_counter() - t
    gm = OSP.to_modal(leg["f32_gN"], q.M, q.dim)[:, sample]
    f32_err = float(np.linalg.norm(gm - refm) / np.linalg.norm(refm))
    ms = statistics.mean(leg["f32_ms"])
    kms = statistics.mean(leg["f32_kernel_ms"])
    f32_flops = (4 * q.np1 + 2) * q.ndof * q.N
    f32 = {
        "workload": "%s fast form: 2D %dx%d (%d DOF), N=%d, BE, alpha=(%g,%g), m=%g, Np=%d"
                    % (PREC_WORKLOAD, q.M, q.M, q.ndof, q.N, q.alpha1, q.alpha2, q.m, q.np1),
        "precision": "FP32 history state and sums, FP64 tables, double-float 2x2 step",
        "value": q.ndof * q.N / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
        "roofline": {"kernel": "k_fp2s_fast_f32", "bound": "alu", "unit": "TFLOP/s",
                     "achieved": f32_flops / (kms * 1e-3) / 1e12, "peak": FP32_PEAK_PROBE / 1e12,
                     "frac": f32_flops / (kms * 1e-3) / FP32_PEAK_PROBE,
                     "peak_source": "own FFMA probe (FP32)", "kernel_ms": kms},
        "error_vs_fp64_oracle_rel_l2_sampled_modes": f32_err, "status": leg["f32_status"],
        "cpu_baseline": {"value": 2 * len(sample) * q.N / t_f, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "oracle FP64 fast BE scheme, %d modes x %d steps (%.1f s)"
                                   % (len(sample), q.N, t_f)},
    }
    return {"tensor_core_direct_history": tc, "tensor_core_direct_history_tf32x3": tf32, "fp32_fast_solve": f32,
            "mixed_direct_solve": mixed_report(leg["mixed"], G0, cpu_modes)}


def mixed_report(runs, G0, cpu_modes):
    """Errors of the mixed-precision direct solves against the FP64 oracle direct scheme
    on sampled modes (the lowest four and a seeded sample), and the main case's rates."""
    import numpy as np
    import cq_inputs as ci
    from oracle import scheme as OS
    from oracle import spatial as OSP
    q0 = runs[0]["problem"]
    nm = q0.M ** q0.dim
    sample = np.unique(np.concatenate([[0, 1, q0.M, q0.M + 1],
                                       ci.sample_indices(nm, max(4, cpu_modes // 8), ci.SEED_BASE + 33)]))
    lam = OSP.mode_eigenvalues(q0.M, q0.dim)[sample]
    g0 = OSP.to_modal(G0, q0.M, q0.dim)[:, sample]
    cases, t_orc, per_step = [], None, None
    for r in runs:
        q = r["problem"]
        t = time.perf_counter()
        traj = OS.solve_modal(q, lam, g0)
        ref = traj[q.N]
        if t_orc is None:
            t_orc = time.perf_counter() - t
        gm = OSP.to_modal(r["gN"], q.M, q.dim)[:, sample]
        err = [float(np.linalg.norm(gm[s] - ref[s]) / np.linalg.norm(ref[s])) for s in range(2)]
        if "partial" in r:
            per_step = {}
            for n, G in sorted(r["partial"].items()):
                gn = OSP.to_modal(G, q.M, q.dim)[:, sample]
                per_step[str(n)] = [float(np.linalg.norm(gn[s] - traj[n][s]) / np.linalg.norm(traj[n][s]))
                                    for s in range(2)]
            per_step[str(q.N)] = err
        cases.append({"scheme": "BE" if q.scheme == ci.BE else "BDF2", "alpha": [q.alpha1, q.alpha2],
                      "contraction": r["prec"],
                      "ms": statistics.mean(r["ms"]), "status": r["status"],
                      "rel_l2_err_vs_fp64_oracle": err})
    main = runs[0]
    q = main["problem"]
    ms = statistics.mean(main["ms"])
    tc_ms = statistics.mean(main["tc_ms"])
    B = 128
    nblk = (q.N + B - 1) // B
    # contraction flops: per block b >= 1, 3 products x 2 x 128 rows x 128 b levels x 2 nm columns
    tc_flops = 3 * 2.0 * B * B * 2 * nm * sum(range(1, nblk))
    peaks = _measured_peaks()
    bf16_peak = peaks.get("bf16_tflops_sustained", 1712.8)
    return {
        "workload": "%s direct form, 2D %dx%d (%d DOF), N=%d, m=%g; BE and BDF2 x alpha in {0.2,0.8}^2"
                    % (PREC_WORKLOAD, q.M, q.M, q.ndof, q.N, q.m),
        "precision": "tensor-core BF16x3 history of earlier 128-step blocks (FP32 accumulation), FP32 in-block "
                     "sums, two-term FP32 step with a double-float amplification matrix",
        "value": q.ndof * q.N / (ms * 1e-3), "unit": UNIT, "ms_per_solve": ms,
        "gpu_launches_per_solve": main["launches"],
        "roofline": {"kernel": "k_history_tc<float, BF16X3> (63 launches per solve)", "bound": "tensor",
                     "unit": "TFLOP/s", "achieved": tc_flops / (tc_ms * 1e-3) / 1e12, "peak": bf16_peak,
                     "frac": tc_flops / (tc_ms * 1e-3) / 1e12 / bf16_peak, "contraction_ms": tc_ms,
                     "share_of_solve": tc_ms / ms,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (kernel inside a long solve)",
                     "algorithmic_flops_per_solve": tc_flops},
        "whole_solve_tensor_equivalent_tflops": 3 * 2.0 * 2 * nm * q.N * (q.N - 1) / 2 / (ms * 1e-3) / 1e12,
        "error_sample": "%d modes (4 lowest + seeded), final step N" % len(sample),
        "rel_l2_err_vs_fp64_oracle_per_step": per_step,
        "per_step_note": "main case (BE, alpha = (0.2, 0.8), BF16x3): level n of the N = 8192 run is the final "
                         "level of the same scheme with N = n and T = n tau",
        "cases": cases,
        "cpu_baseline": {"value": 2 * len(sample) * q.N / t_orc, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "oracle FP64 direct BE scheme, %d modes x %d steps (%.1f s)"
                                   % (len(sample), q.N, t_orc)},
    }


GRAD_WORKLOAD = "grad_2d_m255"


def gradient_leg(fc, torch, dev, K, flush):
    """Gradient of 1/2 ||G^N - G_target||^2 with respect to G0 and (alpha1, alpha2) on the
    2D 255x255 BDF2 workload (N = 4096), target = the same scheme with alpha + (0.05, -0.05);
    dJ/dalpha checked against central differences of the forward solve."""
    import numpy as np
    import cq_inputs as ci
    p, G0 = ci.workload(GRAD_WORKLOAD)

    def cprob(q):
        return fc.problem(q.alpha1, q.alpha2, q.m, q.T, q.N, q.dim, q.M, q.scheme, ci.DIRECT)

    g0 = torch.tensor(G0, dtype=torch.float64, device=dev)
    gt = torch.empty_like(g0)
    wsf = fc.workspace(fc.fp2s_solve(cprob(p), g0, gt, None), dev)
    fc.fp2s_solve(cprob(p.replace(alpha1=p.alpha1 + 0.05, alpha2=p.alpha2 - 0.05)), g0, gt, wsf)
    Gt = gt.cpu().numpy()
    h = 1.0 / (p.M + 1)

    def J_of(q):
        gN = torch.empty_like(g0)
        fc.fp2s_solve(cprob(q), g0, gN, wsf)
        return 0.5 * h ** p.dim * float(np.sum((gN.cpu().numpy() - Gt) ** 2))

    dg = torch.empty_like(g0)
    cp = cprob(p)
    ws = fc.workspace(fc.fp2s_gradient(cp, g0, gt, dg, None), dev)
    J, da = fc.fp2s_gradient(cp, g0, gt, dg, ws)              # warm-up
    times, kern = [], []
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        J, da = fc.fp2s_gradient(cp, g0, gt, dg, ws)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        kern.append(fc.cq_timing_last())
    del ws
    eps = 1e-5
    fd = []
    for f in ("alpha1", "alpha2"):
        v = getattr(p, f)
        fd.append((J_of(p.replace(**{f: v + eps})) - J_of(p.replace(**{f: v - eps}))) / (2 * eps))
    ms = statistics.mean(times)
    rel = [abs(da[i] - fd[i]) / abs(fd[i]) for i in range(2)]
    dG64 = dg.clone()
    mixed = [mixed_gradient_run(fc, torch, dev, p, g0, gt, prec, name, J, da, dG64, fd, ms, 3, flush)
             for name, prec in (("BF16x3", fc.CQ_BF16X3), ("TF32x3", fc.CQ_TF32X3))]
    return {
        "workload": "%s: 2D %dx%d (%d DOF), N=%d, BDF2 direct, alpha=(%g,%g), m=%g; target = same scheme with "
                    "alpha + (0.05,-0.05); J = 1/2 h^2 ||G^N - G_target||^2" % (GRAD_WORKLOAD, p.M, p.M, p.ndof, p.N,
                                                                              p.alpha1, p.alpha2, p.m),
        "precision": "FP64 (forward history kept in full; adjoint of the direct scheme)",
        "value": 1e3 / ms, "unit": "grad steps/s (gradient evaluations per second)", "ms_per_gradient": ms,
        "dof_steps_per_s": p.ndof * p.N / (ms * 1e-3),
        "kernels_ms": statistics.mean(kern), "J": J, "dJ_dalpha": list(da), "fd_dJ_dalpha": fd,
        "rel_err_vs_central_differences": rel, "fd_step": eps,
        "cpu_baseline": None,
        "cpu_baseline_note": "the oracle adjoint is an O(N^2) Python loop; at N = 4096 it exceeds the bench's CPU "
                             "budget, so it is timed only in the tests on small problems",
        "mixed_precision": mixed,
    }


def mixed_gradient_run(fc, torch, dev, p, g0, gt, prec, name, J64, da64, dG64, fd, ms64, K, flush):
    """The same gradient through the mixed-precision direct solve (tensor-core histories on
    FP32 levels): time, contraction roofline, and errors against the FP64 gradient and the
    central differences of the FP64 forward solve."""
    import cq_inputs as ci
    cp = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, ci.DIRECT, prec=prec)
    dg = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_gradient(cp, g0, gt, dg, None), dev)
    Jm, dam = fc.fp2s_gradient(cp, g0, gt, dg, ws)            # warm-up
    times, kern, tcs = [], [], []
    l0 = fc.cq_launch_count()
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        Jm, dam = fc.fp2s_gradient(cp, g0, gt, dg, ws)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        kern.append(fc.cq_timing_last())
        tcs.append(fc.cq_timing_part(1))
    launches = (fc.cq_launch_count() - l0) / K
    del ws
    ms, tc_ms = statistics.mean(times), statistics.mean(tcs)
    nm, N, B = p.M ** p.dim, p.N, 128
    nblk = (N + B - 1) // B
    # contractions: forward and adjoint sweeps (earlier blocks' levels for every block) and the
    # weight-derivative history over all N rows; 3 products x 2 flops x 2 nm columns
    sweep = 3 * 2.0 * B * B * 2 * nm * sum(range(1, nblk))
    flops = 2 * sweep + 3 * 2.0 * 2 * nm * N * (N + 1) / 2
    peaks = _measured_peaks()
    if prec == fc.CQ_TF32X3:
        peak = peaks.get("bf16_tflops_sustained", 1712.8) * 1.1 / 2.25
        peak_src = "MEASURED_PEAKS.json bf16_tflops_sustained x nominal TF32/BF16 ratio 1.1/2.25"
    else:
        peak = peaks.get("bf16_tflops_sustained", 1712.8)
        peak_src = "MEASURED_PEAKS.json bf16_tflops_sustained (kernels inside a long call)"
    dgc, d64 = dg.double(), dG64.double()
    return {
        "precision": "%s contractions on FP32 levels (forward, weight-derivative history of the increments, "
                     "reversed-time adjoint), FP64 weights and step coefficients" % name,
        "value": 1e3 / ms, "unit": "grad steps/s (gradient evaluations per second)", "ms_per_gradient": ms,
        "dof_steps_per_s": p.ndof * p.N / (ms * 1e-3), "kernels_ms": statistics.mean(kern),
        "speedup_vs_fp64_gradient": ms64 / ms,
        "gpu_launches_per_gradient": launches,
        "roofline": {"kernel": "k_history_tc<float, %s> (all contractions of one gradient)" % name.upper(),
                     "bound": "tensor", "unit": "TFLOP/s", "achieved": flops / (tc_ms * 1e-3) / 1e12, "peak": peak,
                     "frac": flops / (tc_ms * 1e-3) / 1e12 / peak, "contraction_ms": tc_ms,
                     "share_of_gradient": tc_ms / ms, "peak_source": peak_src, "algorithmic_flops": flops},
        "J": Jm, "dJ_dalpha": list(dam),
        "rel_err_vs_fp64_gradient": {
            "J": abs(Jm - J64) / abs(J64),
            "dJ_dalpha": [abs(dam[i] - da64[i]) / abs(da64[i]) for i in range(2)],
            "dJ_dG0_rel_l2": float(torch.linalg.norm(dgc - d64) / torch.linalg.norm(d64))},
        "rel_err_vs_central_differences": [abs(dam[i] - fd[i]) / abs(fd[i]) for i in range(2)],
    }


def batch_leg(fc, torch, dev, K, flush):
    """256 independent instances (uneven alpha, m, grid, N, scheme; FP64 fast form) in one
    persistent launch; compared with the same instances solved one call at a time."""
    import numpy as np
    import cq_inputs as ci
    probs, fields, redraws = ci.batch_workload()
    fields = [f * SCALE for f in fields]
    cps = [fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                      flags=fc.FP2S_ASYNC) for p in probs]
    ws = fc.workspace(fc.fp2s_batch_plan(cps), dev)
    t = time.perf_counter()
    plan = fc.fp2s_batch_plan(cps, ws, tune=True)
    plan_s = time.perf_counter() - t
    g0 = torch.tensor(np.concatenate([f.reshape(-1) for f in fields]), dtype=torch.float64, device=dev)
    gN = torch.empty_like(g0)
    fc.fp2s_solve_batched(plan, g0, gN, ws)                       # warm-up
    times, kern = [], []
    l0 = fc.cq_launch_count()
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fc.fp2s_solve_batched(plan, g0, gN, ws)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        kern.append(fc.cq_timing_last())
    launches = (fc.cq_launch_count() - l0) / K
    status = fc.strerror(fc.fp2s_batch_status(plan, ws))
    batch = gN.cpu().numpy()
    del ws
    # the same instances, one fp2s_solve each (same arithmetic per mode)
    singles, t_single, o = [], 0.0, 0
    for cp, f in zip(cps, fields):
        a = torch.tensor(f, dtype=torch.float64, device=dev)
        b = torch.empty_like(a)
        w = fc.workspace(fc.fp2s_solve(cp, a, b, None), dev)
        fc.fp2s_solve(cp, a, b, w)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fc.fp2s_solve(cp, a, b, w)
        e1.record()
        e1.synchronize()
        t_single += e0.elapsed_time(e1)
        n = f.size
        ref = b.cpu().numpy().reshape(-1)
        got = batch[o:o + n]
        o += n
        sc = np.frexp(np.max(np.abs(ref)) if np.max(np.abs(ref)) > 0 else 1.0)[1]
        singles.append(float(np.max(np.abs(np.ldexp(got - ref, -sc)))))
    ms = statistics.mean(times)
    dof_steps = sum(2 * p.M ** p.dim * p.N for p in probs)
    # algorithmic FP64 flops: per DOF-step 4 np + 2 (L - 1) (node recurrences and sums, exact window)
    flops = 0.0
    for p in probs:
        np_, L = (p.np1, 2) if p.scheme == ci.BE else (p.np1 + p.np2, p.ns)
        flops += (4 * np_ + 2 * (L - 1)) * 2.0 * p.M ** p.dim * p.N
    kms = statistics.mean(kern)
    return {
        "workload": "256 seeded instances (alpha ~ U(0.1,0.9), m in [0.30,0.48]U[0.52,0.70], 1D M in [31,1023] "
                    "or 2D M in [31,255] log-uniform, N in [512,8192] log-uniform, BE/BDF2), FP64 fast form, "
                    "G0 = U[0,1) on [1/4,3/4]^d x 2^-1000; %d draws replaced by the growth screen" % redraws,
        "value": dof_steps / (ms * 1e-3), "unit": UNIT, "ms_per_batch": ms, "kernel_ms": statistics.mean(kern),
        "total_dof_steps": dof_steps, "warps_per_block": plan.warps_per_block, "autotuned": bool(plan.flags & 1),
        "plan_s": plan_s, "gpu_launches_per_solve": launches, "status": status,
        "sum_of_single_solves_ms": t_single, "persistent_launch_efficiency": t_single / ms,
        "max_abs_diff_vs_single_solves_rel_to_instance_max": max(singles),
        "roofline": {"kernel": "k_b_fast", "bound": "alu", "unit": "TFLOP/s",
                     "achieved": flops / (kms * 1e-3) / 1e12, "peak": FP64_PEAK_NOMINAL / 1e12,
                     "frac": flops / (kms * 1e-3) / FP64_PEAK_NOMINAL, "peak_source": "nominal FP64 rate (recipe)",
                     "algorithmic_flops_per_launch": flops,
                     "flops_definition": "sum over instances of (4 np + 2 (L - 1)) x DOF x N"},
    }


# The paper's own CPU times (Tables 1 and 5; hardware not stated): context only.
PAPER_TIMES = {"table1": {"BE": 78.53, "FBE": 23.95}, "table5": {"SBD": 870.13, "FSBD": 209.44}}


def small_leg(fc, torch, dev, K):
    """The 1D BE workload (63 interior points, N = 1024, FP64 direct): launch- and
    latency-bound (126 DOF), so only its absolute rate is reported, with its error against
    the oracle over all 63 modes and the oracle's own time."""
    import numpy as np
    import cq_inputs as ci
    from oracle import scheme as OS
    p, G0 = ci.workload("be1d_m63")
    cp = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns)
    g0 = torch.tensor(G0, dtype=torch.float64, device=dev)
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), dev)
    for _ in range(3):
        fc.fp2s_solve(cp, g0, gN, ws)
    times = []
    for _ in range(K):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fc.fp2s_solve(cp, g0, gN, ws)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    got = gN.cpu().numpy()
    t = time.perf_counter()
    ref = OS.solve(p, G0)
    t_orc = time.perf_counter() - t
    ms = statistics.mean(times)
    return {
        "workload": "be1d_m63: 1D, 63 interior points (126 DOF), T=1, N=1024, BE direct FP64, alpha=(0.3,0.7), "
                    "m=0.4, G0 = indicator of [1/4,3/4]",
        "value": p.ndof * p.N / (ms * 1e-3), "unit": UNIT, "ms_per_solve": ms,
        "note": "launch- and latency-bound (the whole history fits in L2); no roofline fraction",
        "rel_l2_err_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
        "cpu_baseline": {"value": p.ndof * p.N / t_orc, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "oracle direct BE scheme, all 63 modes x 1024 steps (%.2f s)" % t_orc},
    }


def paper_leg(fc, torch):
    """Two of the paper's timed runs on the GPU solver: Table 1 (BE / fast BE, h = 1/256,
    1/tau = 1600, alpha = (0.3, 0.6)) and Table 5 (SBD / fast SBD, h = 1/1024, T = 10,
    N = 20000, alpha = (0.3, 0.8)); errors against the plain-scheme reference as in the paper."""
    from paper_1901_05128_gb300 import tables as TB
    out = {}
    for name, alpha, col in (("table1", (0.3, 0.6), -1), ("table5", (0.3, 0.8), 0)):
        ex = dict(TB.EXPERIMENTS[name])
        ex["alphas"] = [alpha]
        ex["inv_tau"] = [ex["inv_tau"][col]]
        key = name + "_bench"
        TB.EXPERIMENTS[key] = ex
        try:
            res = TB.run(key, fc, torch)
        finally:
            del TB.EXPERIMENTS[key]
        row = res["rows"][0]
        labels = ("BE", "FBE") if name == "table1" else ("SBD", "FSBD")
        ndof = 2 * ex["M"]
        N = int(round(ex["inv_tau"][0] * ex["T"]))
        entry = {"grid": "1D, h = 1/%d, N = %d, alpha = %s" % (ex["M"] + 1, N, alpha)}
        for form, lab in zip(("direct", "fast"), labels):
            t = row[form]["gpu_s"][0]
            entry[lab] = {"gpu_s": t, "dof_steps_per_s": ndof * N / t,
                          "E": [float(v) for v in row[form]["E"][0]],
                          "paper_cpu_s": PAPER_TIMES[name][lab]}
        out[name] = entry
    return out


def stream_leg(fc, torch, dev, steps=24):
    """Per-step fast history (cq_history_fast) streaming its state from HBM, FP32 and FP64,
    on the 2D 511x511 DOF count with the BDF2 sizes of the main workload (np = 80, Ns = 17);
    plus the FP32 form on 4 Mi DOFs (a longer kernel: the asymptotic bandwidth)."""
    import cq_inputs as ci
    p, _ = ci.workload(PREC_WORKLOAD)
    out = _stream_case(fc, torch, dev, p.ndof, steps, (("f32", fc.CQ_F32), ("f64", fc.CQ_F64)))
    out.update({k + "_4Mi_dof": v for k, v in _stream_case(fc, torch, dev, 4 << 20, steps, (("f32", fc.CQ_F32),)).items()
                if k != "workload"})
    return out


def _stream_case(fc, torch, dev, ndof, steps, precs):
    import cq_inputs as ci
    np1, np2, ns, beta, tau = 16, 64, 17, 0.6, 1.0 / 4096
    npt = np1 + np2
    gen = torch.Generator(device=dev)
    gen.manual_seed(ci.SEED_BASE + 8)
    G = torch.randn(2, ndof, dtype=torch.float64, device=dev, generator=gen)
    H = torch.empty(ndof, dtype=torch.float64, device=dev)
    out = {}
    per_dofs = {"f32": 8 * npt + 4 * (ns - 2) + 4 + 4 + 8 + 8, "f64": 16 * npt + 8 * (ns - 2) + 8 + 8 + 8 + 8}
    for name, prec in precs:
        per_dof = per_dofs[name]
        ws = fc.workspace(fc.cq_history_fast(2, beta, tau, np1, np2, ns, ndof, 1, None, None, prec=prec), dev)
        n = 1
        for _ in range(ns + 8):                                # past the exact window: full traffic
            fc.cq_history_fast(2, beta, tau, np1, np2, ns, ndof, n, G[n % 2], H, ws, prec=prec)
            n += 1
        torch.cuda.synchronize()
        kms = []
        for _ in range(steps):
            fc.cq_history_fast(2, beta, tau, np1, np2, ns, ndof, n, G[n % 2], H, ws, prec=prec)
            kms.append(fc.cq_timing_last())
            n += 1
        ms = statistics.median(kms)
        bytes_per_launch = per_dof * ndof
        gbs = bytes_per_launch / (ms * 1e-3) / 1e9
        hbm = _measured_peaks().get("hbm_gbs", 6790.0)
        hbm_roof = {"kernel": "k_history_fast_step" + ("_f32" if name == "f32" else ""),
                    "bound": "hbm", "unit": "GB/s", "achieved": gbs, "peak": hbm, "frac": gbs / hbm,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                    "algorithmic_bytes_per_dof_step": per_dof,
                    "algorithmic_bytes_per_launch": bytes_per_launch}
        if name == "f64":
            # 4 flops per node (state update and history FMA) and 2 per exact-window term: at the
            # FP64 rate this takes longer than moving the bytes, so the FP64 pipe is the roof
            flops = (4 * npt + 2 * (ns - 1)) * ndof
            tf = flops / (ms * 1e-3) / 1e12
            roof = {"kernel": "k_history_fast_step", "bound": "alu", "unit": "TFLOP/s", "achieved": tf,
                    "peak": FP64_PEAK_NOMINAL / 1e12, "frac": tf * 1e12 / FP64_PEAK_NOMINAL,
                    "peak_source": "nominal FP64 rate (recipe)", "algorithmic_flops_per_launch": flops,
                    "hbm": hbm_roof,
                    "note": "FP64 time floor %.3f ms vs HBM floor %.3f ms" % (flops / FP64_PEAK_NOMINAL * 1e3,
                                                                             bytes_per_launch / (hbm * 1e9) * 1e3)}
        else:
            roof = hbm_roof
        out[name] = {"value": ndof / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "roofline": roof}
        del ws
    torch.cuda.empty_cache()
    out["workload"] = ("cq_history_fast, one step over %d DOFs, BDF2 sizes np = %d, Ns = %d; "
                       "state %.2f GB (FP32) / %.2f GB (FP64) streamed every step; median of %d steps"
                       % (ndof, npt, ns, npt * ndof * 4 / 1e9, npt * ndof * 8 / 1e9, steps))
    return out


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    import cq_inputs as ci
    import paper_1901_05128_gb300 as pkg

    pkg.build()
    fc = pkg.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    p, G0 = ci.workload(WORKLOAD)
    if rank:
        G0 = ci.g0_checkerboard_uniform(p.M, ci.SEED_BASE + 1 + 1000 * rank)
    G0 = G0 * SCALE
    flags = fc.FP2S_ASYNC

    def cproblem(q):
        return fc.problem(q.alpha1, q.alpha2, q.m, q.T, q.N, q.dim, q.M, q.scheme, q.form, q.np1, q.np2, q.ns,
                          flags=flags)

    g0 = torch.tensor(G0, dtype=torch.float64, device=dev)
    gN = torch.empty_like(g0)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MiB > 2x L2
    fc.cq_timing_enable(True)

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(q, K, W):
        cp = cproblem(q)
        ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), dev)
        for _ in range(W):
            fc.fp2s_solve(cp, g0, gN, ws)
        st = fc.fp2s_status(cp, ws)
        if st not in (fc.CQ_OK,):
            raise RuntimeError("warm-up solve failed: %s" % fc.strerror(st))
        barrier()
        torch.cuda.synchronize()
        l0 = fc.cq_launch_count()
        steps, mains = [], []
        for _ in range(K):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fc.fp2s_solve(cp, g0, gN, ws)
            e1.record()
            e1.synchronize()
            steps.append(e0.elapsed_time(e1))
            mains.append(fc.cq_timing_last())
        torch.cuda.synchronize()
        barrier()
        launches = fc.cq_launch_count() - l0
        st = fc.fp2s_status(cp, ws)
        return steps, mains, launches, st

    K, W = args.steps, args.warmup
    with ClockSampler(torch.cuda.current_device()) as clk:
        steps, mains, launches, st_fast = timed(p, K, W)
        gN_fast = gN.cpu().numpy()
        pd = p.replace(form=ci.DIRECT)
        Kd, Wd = max(1, min(K, 4)), max(1, min(W, 1))
        d_steps, d_mains, d_launches, st_dir = timed(pd, Kd, Wd)
        gN_dir = gN.cpu().numpy()
        # end to end through the public API with pinned host buffers
        cp = cproblem(p)
        ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), dev)
        h_in = torch.tensor(G0, dtype=torch.float64).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        fc.fp2s_solve(cp, g0, gN, ws)
        barrier()
        torch.cuda.synchronize()
        e2e = []
        for _ in range(K):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g0.copy_(h_in, non_blocking=True)
            fc.fp2s_solve(cp, g0, gN, ws)
            h_out.copy_(gN, non_blocking=True)
            e1.record()
            e1.synchronize()
            e2e.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier()
        del ws
        prec_leg = precision_leg(fc, torch, dev, max(1, min(K, 3)), 1, flush) if (args.precision and rank == 0) \
            else None
        grad = gradient_leg(fc, torch, dev, 2, flush) if (args.precision and rank == 0) else None
        batch = batch_leg(fc, torch, dev, 2, flush) if (args.precision and rank == 0) else None
        stream = stream_leg(fc, torch, dev) if (args.precision and rank == 0) else None
        paper = paper_leg(fc, torch) if (args.precision and rank == 0) else None
        small = small_leg(fc, torch, dev, 10) if (args.precision and rank == 0) else None
    clocks = clk.summary()

    ms = statistics.mean(steps)
    ms_main = statistics.mean(mains)
    ms_dir = statistics.mean(d_steps)
    ms_e2e = statistics.mean(e2e)
    if dist is not None:
        t = torch.tensor([ms, ms_dir, ms_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_dir, ms_e2e = t.tolist()
    units = p.ndof * p.N
    value = world * units / (ms * 1e-3)
    if rank != 0:
        return None

    # roofline of the dominant kernel (fused fast solve): FP64-pipe bound
    hist_flops_per_dof_step = 4 * (p.np1 + p.np2) + 2 * (p.ns - 1)
    flops_per_launch = hist_flops_per_dof_step * units
    achieved = flops_per_launch / (ms_main * 1e-3)
    roofline = {"kernel": "k_fp2s_fast", "bound": "alu", "unit": "TFLOP/s",
                "achieved": achieved / 1e12, "peak": FP64_PEAK_NOMINAL / 1e12,
                "frac": achieved / FP64_PEAK_NOMINAL, "peak_source": "nominal FP64 rate (recipe); own DFMA probe "
                "measured %.3f TFLOP/s" % (FP64_PEAK_PROBE / 1e12),
                "traffic": None, "algorithmic_flops_per_launch": flops_per_launch,
                "flops_per_dof_step": hist_flops_per_dof_step, "kernel_ms": ms_main,
                "kernel_share_of_step": ms_main / ms}
    traffic = _profiled_traffic("k_fp2s_fast_bdf2_2d_m255.md")
    if traffic is not None:
        roofline["traffic"] = traffic
        roofline["traffic_note"] = "ncu dram bytes per launch (independent of N: state stays on chip)"

    # oracle leg: bounded sample, also gives the error of this run
    import numpy as np
    from oracle import spatial as OSP
    sample, ref_fast, t_fast = oracle_sample(p, G0, args.cpu_modes, ci.SEED_BASE + 21)
    sample_d, ref_dir, t_dir = oracle_sample(p.replace(form=ci.DIRECT), G0, max(4, args.cpu_modes // 16),
                                             ci.SEED_BASE + 22)

    def scaled(x, ref):
        # exact power-of-two rescaling (values span ~1e-300..1e+176 here) before any norm
        e = np.frexp(np.max(np.abs(ref)))[1]
        return np.ldexp(x, -e), np.ldexp(ref, -e)

    def rel_err(gN_phys, sample_idx, ref):
        # max error over the sampled modes relative to the largest sampled mode: the
        # comparison goes through one extra DST, which adds ~eps * max|g| to every mode
        ghat = OSP.to_modal(gN_phys, p.M, p.dim)[:, sample_idx]
        g, r = scaled(ghat, ref)
        return float(np.max(np.abs(g - r)) / np.max(np.abs(r)))

    err_fast = rel_err(gN_fast, sample, ref_fast)
    err_dir = rel_err(gN_dir, sample_d, ref_dir)
    mf, md = scaled(OSP.to_modal(gN_fast, p.M, p.dim), OSP.to_modal(gN_dir, p.M, p.dim))
    fast_vs_direct = float(np.linalg.norm(mf - md) / np.linalg.norm(md))
    cpu_value = 2 * len(sample) * p.N / t_fast

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; see config)", "config": workload_config(p),
        "roofline": roofline,
        "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
                         "sample": "oracle fast SBD scheme, %d seeded sine modes x all %d steps (%.1f s)"
                                   % (len(sample), p.N, t_fast)},
        "e2e": {"value": world * units / (ms_e2e * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(G0.size * 8), "d2h_bytes_per_step": int(G0.size * 8),
                "ms_per_step": ms_e2e},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "error": {"fast_vs_oracle_max_err_rel_to_max_mode": err_fast,
                  "direct_vs_oracle_max_err_rel_to_max_mode": err_dir,
                  "fast_vs_direct_rel_l2": fast_vs_direct, "status": fc.strerror(st_fast)},
        "direct": {"value": world * units / (ms_dir * 1e-3), "unit": UNIT, "ms_per_step": ms_dir, "steps": Kd,
                   "warmup": Wd, "kernel": "k_fp2s_direct<8>", "kernel_ms": statistics.mean(d_mains),
                   "gpu_launches": int(d_launches), "status": fc.strerror(st_dir),
                   "cpu_baseline": {"value": 2 * len(sample_d) * p.N / t_dir, "unit": UNIT, "cores": 1,
                                    "kind": "oracle", "sample": "oracle direct SBD scheme, %d modes x %d steps "
                                    "(%.1f s)" % (len(sample_d), p.N, t_dir)}},
        "device": torch.cuda.get_device_name(),
    }
    if prec_leg is not None:
        out["precision"] = precision_report(prec_leg, max(16, args.cpu_modes // 64))
    if grad is not None:
        out["gradient"] = grad
    if batch is not None:
        out["batch"] = batch
    if stream is not None:
        out["fast_history_stream"] = stream
    if paper is not None:
        out["paper_runs"] = {"note": "the paper's CPU times are on unstated hardware: context only", **paper}
    if small is not None:
        out["small_1d"] = small
    return out


def _kernel_hash():
    """Hash of the source of k_fp2s_fast (its function text in fp2s.cu) and of the headers it
    uses: a traffic figure recorded under another hash was taken on another kernel."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1901_05128_gb300", "csrc")
    with open(os.path.join(csrc, "fp2s.cu")) as fh:
        src = fh.read()
    i = src.index(" k_fp2s_fast(Fp2sParams P")
    h.update(src[src.rindex("__global__", 0, i):src.index("\n}\n", i) + 3].encode())
    for f in ("fp2s_core.cuh", "common.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(name):
    """DRAM bytes per launch recorded in a profiles/ summary, if it was taken on the current kernel source."""
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch: (\d+) \(source hash ([0-9a-f]+)\)", txt)
    if not m or m.group(2) != _kernel_hash():
        return None
    return int(m.group(1))


# ----------------------------------------------------------------------------- reference arm (the oracle)
def run_reference(args, rank, world):
    if rank != 0:
        return None
    import cq_inputs as ci
    p, G0 = ci.workload(WORKLOAD)
    G0 = G0 * SCALE
    n = args.ref_modes
    for w in range(args.warmup):
        oracle_sample(p.replace(N=64, T=p.T * 64 / p.N), G0, n, ci.SEED_BASE + 30 + w)
    times = []
    for k in range(args.steps):
        _, _, dt = oracle_sample(p, G0, n, ci.SEED_BASE + 40 + k)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = 2 * n * p.N / (ms * 1e-3)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; see config)",
            "config": workload_config(p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
                             "sample": "each step: oracle fast SBD scheme on %d seeded sine modes x all %d steps "
                                       "(warm-up steps use N=64)" % (n, p.N)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-modes", type=int, default=8192, help="sine modes of the oracle's timed sample")
    ap.add_argument("--ref-modes", type=int, default=2048, help="sine modes per step of the reference arm")
    ap.add_argument("--no-precision", dest="precision", action="store_false",
                    help="leave out the precision-form, gradient and batch legs")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "ours":
        import torch
        if world > 1:
            import torch.distributed as tdist
            local = int(os.environ.get("LOCAL_RANK", "0"))
            torch.cuda.set_device(local)
            tdist.init_process_group("nccl")
            dist = tdist
        out = run_ours(args, rank, world, dist)
        if dist is not None:
            dist.destroy_process_group()
    else:
        out = run_reference(args, rank, world)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
