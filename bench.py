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

# Every oracle process does its numpy work on one thread: the one-thread figures use one core,
# and the all-core figures run one spawned process per core (set before numpy is first imported,
# and inherited by the spawned processes).
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
FP32_PEAK_PROBE = 73.2e12         # FP32 FMA probe figure of an earlier run (used only if the probe cannot run)
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


def mode_jobs(p, G0, n_modes, seeds):
    """One oracle job per seed: the per-mode scheme of p on n_modes seeded sine modes."""
    import numpy as np
    from oracle import spatial as OSP
    import cq_inputs as ci
    nm = p.M ** p.dim
    lam_all = OSP.mode_eigenvalues(p.M, p.dim)
    g0_all = OSP.to_modal(G0, p.M, p.dim)
    jobs = []
    for sd in seeds:
        idx = np.sort(ci.sample_indices(nm, min(n_modes, nm), sd))
        jobs.append(("modes", p, lam_all[idx], g0_all[:, idx]))
    return jobs


def _oracle_job(job):
    """One oracle computation (in a spawned worker process, or in this process); returns its
    wall time in seconds. Jobs: ("modes", problem, lam, g0) the per-mode scheme;
    ("history", scheme, beta, tau, G) the direct history of DOF columns; ("gradient",
    problem, G0, Gt) the discrete adjoint gradient; ("warm",) imports only."""
    kind = job[0]
    if kind == "warm":
        from oracle import adjoint, history, scheme  # noqa: F401
        return 0.0
    t = time.perf_counter()
    if kind == "modes":
        from oracle import scheme as OS
        OS.solve_modal(job[1], job[2], job[3])
    elif kind == "history":
        from oracle import history as OH
        from oracle import weights as OW
        G = job[4]
        OH.history_direct_all(OW.weights(job[1], job[2], job[3], G.shape[0]), G, 1, G.shape[0])
    elif kind == "gradient":
        from oracle import adjoint as AD
        AD.gradient(job[1], job[2], job[3])
    else:
        raise ValueError(kind)
    return time.perf_counter() - t


_POOL = None


def _oracle_pool():
    """A pool of one spawned process per host core (spawn: safe after CUDA is initialised),
    warmed up so that the timed maps do not include interpreter start-up and imports."""
    global _POOL
    if _POOL is None:
        import multiprocessing as mp
        n = os.cpu_count() or 1
        _POOL = mp.get_context("spawn").Pool(n)
        _POOL.map(_oracle_job, [("warm",)] * (4 * n), chunksize=1)
    return _POOL


def _close_pool():
    global _POOL
    if _POOL is not None:
        _POOL.close()
        _POOL.join()
        _POOL = None


def _ncpu():
    return os.cpu_count() or 1


def cpu_info():
    """Host cores and CPU model (from /proc/cpuinfo: model name, or the Arm implementer / part)."""
    model = None
    try:
        txt = open("/proc/cpuinfo").read()
        for key in ("model name", "Model Name", "Processor"):
            for line in txt.splitlines():
                if line.split(":")[0].strip() == key:
                    model = line.split(":", 1)[1].strip()
                    break
            if model:
                break
        if not model:
            fields = {}
            for line in txt.splitlines():
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip(), v.strip())
            if "CPU implementer" in fields:
                model = "Arm implementer %s part %s" % (fields.get("CPU implementer"), fields.get("CPU part"))
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count() or 1, "model": model or platform.processor() or platform.machine()}


def cpu_baseline(unit, units_one, t_one, sample_one, jobs_all=None, units_all=None, sample_all=None):
    """The oracle's rate on the host: on every core (one spawned process per core running
    jobs_all, wall time of the whole map) with the one-thread figure beside it (units_one
    units of work in t_one seconds on one core)."""
    one = {"value": units_one / t_one, "unit": unit, "cores": 1, "seconds": t_one, "sample": sample_one}
    info = cpu_info()
    out = {"kind": "oracle", "unit": unit, "one_thread": one, "cpu_model": info["model"], "nproc": info["nproc"]}
    if jobs_all:
        pool = _oracle_pool()
        t = time.perf_counter()
        pool.map(_oracle_job, jobs_all, chunksize=1)
        wall = time.perf_counter() - t
        out.update({"value": units_all / wall, "cores": info["nproc"], "seconds": wall,
                    "sample": "%s (%d jobs over %d processes, one per core)" % (sample_all, len(jobs_all),
                                                                              info["nproc"])})
    else:
        out.update({"value": one["value"], "cores": 1, "seconds": t_one, "sample": sample_one})
    return out


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
        "error_vs_oracle": {"max_abs_err_over_sum_abs_terms": tc_err,
                            "bound": 3 * 2.0 ** -16 + 24 * 2.0 ** -23 + (-(-rows // 128)) * 2.0 ** -24,
                            "sample": "%d whole DOF columns x %d steps" % (PREC_COLS, rows)},
        "gpu_launches_per_call": leg["tc_launches"] / max(1, len(leg["tc_gemm_ms"])),
        "cpu_baseline": cpu_baseline(
            UNIT, PREC_COLS * rows, t_orc, "oracle direct history of %d DOF columns x %d steps" % (PREC_COLS, rows),
            [("history", ci.BE, leg["tc_beta"], leg["tc_tau"], ci.rng(ci.SEED_BASE + 50 + k).standard_normal(
                (n_hi, PREC_COLS))) for k in range(_ncpu())],
            _ncpu() * PREC_COLS * rows, "oracle direct history of %d synthetic DOF columns x %d steps per job"
            % (PREC_COLS, rows)),
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
                     "achieved": f32_flops / (kms * 1e-3) / 1e12, "peak": alu_peak("fp32")[0] / 1e12,
                     "frac": f32_flops / (kms * 1e-3) / alu_peak("fp32")[0],
                     "peak_source": alu_peak("fp32")[1], "kernel_ms": kms,
                     "traffic": _recorded_traffic("k_fp2s_fast_f32"),
                     "flops_definition": "(4 np + 2) per DOF-step (node recurrences, history sums, C G^{n-L}); "
                                         "the double-float remainders of the slow nodes and weights are not counted"},
        "error_vs_fp64_oracle_rel_l2_sampled_modes": f32_err, "status": leg["f32_status"],
        "cpu_baseline": cpu_baseline(
            UNIT, 2 * len(sample) * q.N, t_f, "oracle FP64 fast BE scheme, %d modes x %d steps" % (len(sample), q.N),
            mode_jobs(q, G0, len(sample), [ci.SEED_BASE + 60 + k for k in range(_ncpu())]),
            _ncpu() * 2 * len(sample) * q.N, "oracle FP64 fast BE scheme, %d seeded modes x %d steps per job"
            % (len(sample), q.N)),
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
        "cpu_baseline": cpu_baseline(
            UNIT, 2 * len(sample) * q.N, t_orc, "oracle FP64 direct BE scheme, %d modes x %d steps"
            % (len(sample), q.N),
            mode_jobs(q, G0, len(sample), [ci.SEED_BASE + 70 + k for k in range(_ncpu())]),
            _ncpu() * 2 * len(sample) * q.N, "oracle FP64 direct BE scheme, %d seeded modes x %d steps per job"
            % (len(sample), q.N)),
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
    df = mixed_gradient_run(fc, torch, dev, p, g0, gt, fc.CQ_DF64, "DF64", J, da, dG64, fd, ms, K, flush)
    df["precision"] = ("double-float (FP32 pairs) weights, stored levels and histories of the forward and "
                       "adjoint sweeps; FP64 2x2 steps")
    fast = fast_gradient_run(fc, torch, dev, p, g0, gt, Gt, K, flush, da, dG64, ms, J)
    return {
        "workload": "%s: 2D %dx%d (%d DOF), N=%d, BDF2 direct, alpha=(%g,%g), m=%g; target = same scheme with "
                    "alpha + (0.05,-0.05); J = 1/2 h^2 ||G^N - G_target||^2" % (GRAD_WORKLOAD, p.M, p.M, p.ndof, p.N,
                                                                              p.alpha1, p.alpha2, p.m),
        "precision": "FP64 (forward history kept in full; adjoint of the direct scheme)",
        "value": 1e3 / ms, "unit": "grad steps/s (gradient evaluations per second)", "ms_per_gradient": ms,
        "dof_steps_per_s": p.ndof * p.N / (ms * 1e-3),
        "kernels_ms": statistics.mean(kern), "J": J, "dJ_dalpha": list(da), "fd_dJ_dalpha": fd,
        "rel_err_vs_central_differences": rel, "fd_step": eps,
        "cpu_baseline": gradient_cpu_baseline(p),
        "mixed_precision": mixed,
        "df64": df,
        "fast": fast,
    }


def fast_gradient_run(fc, torch, dev, p, g0, gt, Gt, K, flush, da64, dG64, ms64, J64):
    """The same gradient through the fast scheme (FP64, np1/np2/Ns of the workload): time,
    dJ/dalpha against central differences of the fast forward solve, and the distance from the
    direct scheme's gradient (the fast-vs-direct quadrature error)."""
    import numpy as np
    import cq_inputs as ci

    def cprob(q):
        return fc.problem(q.alpha1, q.alpha2, q.m, q.T, q.N, q.dim, q.M, q.scheme, ci.FAST, q.np1, q.np2, q.ns)

    h = 1.0 / (p.M + 1)
    cp = cprob(p)
    dg = torch.empty_like(g0)
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
    # the same with the backward sweep in double-float
    cpd = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, ci.FAST, p.np1, p.np2, p.ns,
                     prec=fc.CQ_DF64)
    dgd = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_gradient(cpd, g0, gt, dgd, None), dev)
    Jd, dad = fc.fp2s_gradient(cpd, g0, gt, dgd, ws)          # warm-up
    dtimes, dkern = [], []
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        Jd, dad = fc.fp2s_gradient(cpd, g0, gt, dgd, ws)
        e1.record()
        e1.synchronize()
        dtimes.append(e0.elapsed_time(e1))
        dkern.append(fc.cq_timing_last())
    del ws
    wsf = fc.workspace(fc.fp2s_solve(cp, g0, gt, None), dev)

    def J_of(q):
        gN = torch.empty_like(g0)
        fc.fp2s_solve(cprob(q), g0, gN, wsf)
        return 0.5 * h ** p.dim * float(np.sum((gN.cpu().numpy() - Gt) ** 2))

    eps = 1e-5
    fd = [(J_of(p.replace(**{f: getattr(p, f) + eps})) - J_of(p.replace(**{f: getattr(p, f) - eps}))) / (2 * eps)
          for f in ("alpha1", "alpha2")]
    ms = statistics.mean(times)
    kms = statistics.mean(kern)
    dG = dg.cpu().numpy()
    d64 = dG64.cpu().numpy()
    npts = p.np1 + p.np2
    # FP64 flops per DOF-step: forward 4 np + 2 (Ns - 1); backward sweep 10 np + 4 (Ns - 1) (per node
    # the V and W recurrences, the d-history and the two d'-history terms; the window of d and d')
    flops = (14.0 * npts + 6.0 * (p.ns - 1)) * p.ndof * p.N
    pk, pk_src = alu_peak("fp64")
    return {
        "precision": "FP64, fast form (np1=%d, np2=%d, Ns=%d): forward fast solve keeping every level, then "
                     "backward geometric recurrences per quadrature node" % (p.np1, p.np2, p.ns),
        "value": 1e3 / ms, "unit": "grad steps/s (gradient evaluations per second)", "ms_per_gradient": ms,
        "kernels_ms": kms, "speedup_vs_direct_fp64_gradient": ms64 / ms, "J": J, "dJ_dalpha": list(da),
        "fd_dJ_dalpha": fd, "rel_err_vs_central_differences": [abs(da[i] - fd[i]) / abs(fd[i]) for i in range(2)],
        "rel_diff_vs_direct_gradient": {"dJ_dalpha": [abs(da[i] - da64[i]) / abs(da64[i]) for i in range(2)],
                                        "dJ_dG0_rel_l2": float(np.linalg.norm(dG - d64) / np.linalg.norm(d64)),
                                        "J_fast_over_J_direct": J / J64,
                                        "note": "the gradient of the fast scheme, exact for that scheme (central "
                                                "differences above); the misfit's residual is small (the target "
                                                "is a nearby solve), so the fast-vs-direct difference of the "
                                                "solutions shows in J and in the gradients"},
        "roofline": {"kernel": "k_fp2s_fast<true> + k_adjoint_fast", "bound": "alu", "unit": "TFLOP/s",
                     "achieved": flops / (kms * 1e-3) / 1e12, "peak": pk / 1e12, "frac": flops / (kms * 1e-3) / pk,
                     "peak_source": pk_src, "algorithmic_flops_per_gradient": flops,
                     "flops_definition": "(14 np + 6 (Ns - 1)) per DOF-step: forward 4 np + 2 (Ns - 1), backward "
                                         "10 np + 4 (Ns - 1)"},
        "cpu_baseline": "the gradient leg's (the oracle's direct adjoint; the fast scheme's oracle gradient runs "
                        "the same O(N^2) recursion with the quadrature weights)",
        "df64": {"precision": "forward and backward sweeps in double-float (FP32 pairs, packed two-wide; FP64 "
                              "steps, stored levels and per-mode sums)",
                 "ms_per_gradient": statistics.mean(dtimes), "kernels_ms": statistics.mean(dkern),
                 "speedup_vs_fp64_fast_gradient": ms / statistics.mean(dtimes),
                 "rel_err_vs_central_differences": [abs(dad[i] - fd[i]) / abs(fd[i]) for i in range(2)],
                 "rel_diff_vs_fp64_fast_gradient": {
                     "J": abs(Jd - J) / abs(J), "dJ_dalpha": [abs(dad[i] - da[i]) / abs(da[i]) for i in range(2)],
                     "dJ_dG0_rel_l2": float(np.linalg.norm(dgd.cpu().numpy() - dG) / np.linalg.norm(dG))}},
    }


def gradient_cpu_baseline(p):
    """The oracle's discrete adjoint (forward scheme, reversed-time adjoint, dJ/dalpha) on a
    bounded sample of the gradient workload: the same scheme, alpha, m and tau on a 15 x 15 grid
    over the first 1024 steps (the direct gradient is O(N^2) per mode, with Python loops over the
    step pairs: the full 4096-step problem would take minutes). One gradient on one core, and one
    per core at once."""
    import cq_inputs as ci
    from oracle import scheme as OS
    q = p.replace(M=15, N=1024, T=p.T * 1024 / p.N)
    tgt = OS.solve(q.replace(alpha1=q.alpha1 + 0.05, alpha2=q.alpha2 - 0.05), ci.g0_checkerboard_uniform(15, 1))
    jobs = [("gradient", q, ci.g0_checkerboard_uniform(15, ci.SEED_BASE + 90 + k), tgt) for k in range(_ncpu())]
    t1 = _oracle_job(jobs[0])
    units = q.ndof * q.N
    desc = "oracle adjoint gradient, 2D 15x15 (%d DOF), first %d steps at tau = 1/%d, BDF2 direct" % (
        q.ndof, q.N, p.N)
    out = cpu_baseline(UNIT, units, t1, desc + ": one gradient", jobs, len(jobs) * units,
                       desc + ", one gradient per job")
    out["grad_steps_per_s"] = {"one_thread": 1.0 / t1, "all_cores": out["value"] / units,
                               "note": "gradients of the sample problem per second"}
    return out


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
    if prec == fc.CQ_DF64:
        # double-float histories on the FP32 pipe: 12 operations per term; forward N^2 / 2 terms per
        # mode and state, adjoint twice that (the d and d' histories)
        ops = 12.0 * 2 * nm * N * N / 2 * 3
        pk, pk_src = alu_peak("fp32")
        roof = {"kernel": "k_fp2s_direct_df<8> + k_adjoint_direct_df<4>", "bound": "alu", "unit": "T FP32-op/s",
                "achieved": ops / (statistics.mean(kern) * 1e-3) / 1e12, "peak": pk / 2e12,
                "frac": ops / (statistics.mean(kern) * 1e-3) / (pk / 2), "peak_source": pk_src + " / 2",
                "fp32_ops": ops}
    else:
        roof = {"kernel": "k_history_tc<float, %s> (all contractions of one gradient)" % name.upper(),
                "bound": "tensor", "unit": "TFLOP/s", "achieved": flops / (tc_ms * 1e-3) / 1e12, "peak": peak,
                "frac": flops / (tc_ms * 1e-3) / 1e12 / peak, "contraction_ms": tc_ms,
                "share_of_gradient": tc_ms / ms, "peak_source": peak_src, "algorithmic_flops": flops}
    return {
        "precision": "%s contractions on FP32 levels (forward, weight-derivative history of the increments, "
                     "reversed-time adjoint), FP64 weights and step coefficients" % name,
        "value": 1e3 / ms, "unit": "grad steps/s (gradient evaluations per second)", "ms_per_gradient": ms,
        "dof_steps_per_s": p.ndof * p.N / (ms * 1e-3), "kernels_ms": statistics.mean(kern),
        "speedup_vs_fp64_gradient": ms64 / ms,
        "gpu_launches_per_gradient": launches,
        "roofline": roof,
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
    # the same solve captured once in a CUDA graph and replayed (no host work per replay)
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        with torch.cuda.graph(graph, stream=gs):
            fc.fp2s_solve_batched(plan, g0, gN, ws)
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    replay = []
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        e1.synchronize()
        replay.append(e0.elapsed_time(e1))
    replay_same = bool(np.array_equal(gN.cpu().numpy(), batch))
    del graph
    del ws
    df64 = batch_df64(fc, torch, dev, K, flush, probs, g0, batch, ms_fp64=statistics.mean(times))
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
    # oracle: a seeded 16-instance subset, each on a seeded sample of at most 64 sine modes x all its steps
    from oracle import spatial as OSP
    pick = ci.sample_indices(len(probs), 16, ci.SEED_BASE + 95)
    jobs, units_each = [], []
    for k, i in enumerate(pick):
        q, f = probs[i], fields[i]
        jobs += mode_jobs(q, f, 64, [ci.SEED_BASE + 96 + k])
        units_each.append(2 * min(64, q.M ** q.dim) * q.N)
    t1 = sum(_oracle_job(j) for j in jobs)
    reps = max(1, -(-2 * _ncpu() // len(jobs)))
    jobs_all = [(j[0], j[1], j[2], j[3]) for _ in range(reps) for j in jobs]
    cpu = cpu_baseline(UNIT, sum(units_each), t1, "oracle FP64 fast scheme, seeded 16-instance subset, <= 64 "
                       "seeded modes per instance x all its steps", jobs_all, reps * sum(units_each),
                       "the same 16 instance samples, %d times over" % reps)
    return {
        "workload": "256 seeded instances (alpha ~ U(0.1,0.9), m in [0.30,0.48]U[0.52,0.70], 1D M in [31,1023] "
                    "or 2D M in [31,255] log-uniform, N in [512,8192] log-uniform, BE/BDF2), FP64 fast form, "
                    "G0 = U[0,1) on [1/4,3/4]^d x 2^-1000; %d draws replaced by the growth screen" % redraws,
        "value": dof_steps / (ms * 1e-3), "unit": UNIT, "ms_per_batch": ms, "kernel_ms": statistics.mean(kern),
        "total_dof_steps": dof_steps,
        "graph_replay": {"value": dof_steps / (statistics.mean(replay) * 1e-3), "unit": UNIT,
                         "ms_per_batch": statistics.mean(replay), "same_result_as_direct_calls": replay_same,
                         "note": "fp2s_solve_batched captured once in a CUDA graph (five kernels, one memset), "
                                 "replayed; L2 flushed before every replay, outside the events"},
        "launch_shape": {"warps_per_block": plan.warps_per_block, "ctas_per_sm": plan.ctas_per_sm or "all that fit",
                         "node_unroll": plan.node_unroll,
                         "autotuned": bool(plan.flags & 1), "candidates_timed": plan.tuned_candidates,
                         "tuner": "block widths 2..16 warps x (all, half of the CTAs per SM that fit) x node-loop "
                                  "width (2, 4, 8 partial sums), 96-step run, median of three timings each"},
        "plan_s": plan_s, "gpu_launches_per_solve": launches, "status": status,
        "sum_of_single_solves_ms": t_single, "persistent_launch_efficiency": t_single / ms,
        "max_abs_diff_vs_single_solves_rel_to_instance_max": max(singles),
        "roofline": {"kernel": "k_b_fast", "bound": "alu", "unit": "TFLOP/s",
                     "achieved": flops / (kms * 1e-3) / 1e12, "peak": alu_peak("fp64")[0] / 1e12,
                     "frac": flops / (kms * 1e-3) / alu_peak("fp64")[0], "peak_source": alu_peak("fp64")[1],
                     "algorithmic_flops_per_launch": flops,
                     "flops_definition": "sum over instances of (4 np + 2 (L - 1)) x DOF x N"},
        "cpu_baseline": cpu,
        "df64": df64,
    }


def batch_df64(fc, torch, dev, K, flush, probs, g0, batch_fp64, ms_fp64):
    """The same 256 instances as one double-float batch (CQ_DF64 for every instance): time per
    batch and the largest difference from the FP64 batch per instance, relative to the instance's
    largest value."""
    import numpy as np
    cps = [fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                      prec=fc.CQ_DF64, flags=fc.FP2S_ASYNC) for p in probs]
    ws = fc.workspace(fc.fp2s_batch_plan(cps), dev)
    plan = fc.fp2s_batch_plan(cps, ws)
    gN = torch.empty_like(g0)
    fc.fp2s_solve_batched(plan, g0, gN, ws)                       # warm-up
    times, kern = [], []
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
    status = fc.strerror(fc.fp2s_batch_status(plan, ws))
    got = gN.cpu().numpy()
    del ws
    worst, o = 0.0, 0
    for p in probs:
        n = 2 * p.M ** p.dim
        a, b = got[o:o + n], batch_fp64[o:o + n]
        o += n
        sc = np.max(np.abs(b))
        if sc > 0:
            worst = max(worst, float(np.max(np.abs(a - b)) / sc))
    ms = statistics.mean(times)
    dof_steps = sum(2 * p.M ** p.dim * p.N for p in probs)
    return {"value": dof_steps / (ms * 1e-3), "unit": UNIT, "ms_per_batch": ms, "kernel_ms": statistics.mean(kern),
            "speedup_vs_fp64_batch": ms_fp64 / ms, "status": status,
            "max_abs_diff_vs_fp64_batch_rel_to_instance_max": worst,
            "kernel": "k_b_df (double-float node states and sums, FP64 step; 64-mode units)"}


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
        "cpu_baseline": cpu_baseline(
            UNIT, p.ndof * p.N, t_orc, "oracle direct BE scheme, all 63 modes x 1024 steps",
            mode_jobs(p, G0, p.M, [ci.SEED_BASE + 80 + k for k in range(4 * _ncpu())]),
            4 * _ncpu() * p.ndof * p.N, "oracle direct BE scheme, all 63 modes x 1024 steps per job"),
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
    """Per-step fast history (cq_history_fast) streaming its state from HBM, FP32, FP64 and double-float,
    on the 2D 511x511 DOF count with the BDF2 sizes of the main workload (np = 80, Ns = 17);
    plus the FP32 and double-float forms on 4 Mi DOFs (a longer kernel: the asymptotic bandwidth)."""
    import cq_inputs as ci
    p, _ = ci.workload(PREC_WORKLOAD)
    out = _stream_case(fc, torch, dev, p.ndof, steps, (("f32", fc.CQ_F32), ("f64", fc.CQ_F64), ("df64", fc.CQ_DF64)))
    out.update({k + "_4Mi_dof": v for k, v in _stream_case(fc, torch, dev, 4 << 20, steps,
                                                          (("f32", fc.CQ_F32), ("df64", fc.CQ_DF64))).items()
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
    per_dofs = {"f32": 8 * npt + 4 * (ns - 2) + 4 + 4 + 8 + 8, "f64": 16 * npt + 8 * (ns - 2) + 8 + 8 + 8 + 8,
                "df64": 16 * npt + 8 * (ns - 2) + 8 + 8 + 8 + 8}
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
        hbm_roof = {"kernel": "k_history_fast_step" + {"f32": "_f32", "df64": "_df"}.get(name, ""),
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
                    "peak": alu_peak("fp64")[0] / 1e12, "frac": tf * 1e12 / alu_peak("fp64")[0],
                    "peak_source": alu_peak("fp64")[1], "algorithmic_flops_per_launch": flops,
                    "hbm": hbm_roof,
                    "note": "FP64 time floor %.3f ms vs HBM floor %.3f ms" % (flops / alu_peak("fp64")[0] * 1e3,
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


_ALU = {}


def fma_peaks(torch, dev):
    """FP64 and FP32 FMA rates of this GPU from the probe library (libcqprobe.so, built with the
    package): 8 CTAs of 256 threads per SM, 8 independent FMA chains per thread, ~50 ms per
    timed launch. They are the ALU roofs of the fast solves (the measured copy and GEMM peaks
    cover HBM and the tensor pipe)."""
    import ctypes as C
    import importlib
    B = importlib.import_module("paper_1901_05128_gb300.build")
    lib = C.CDLL(B.PROBE_LIB)
    f = lib.cq_probe_fma_rate
    f.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    f.restype = C.c_int
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * sms, 256
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    res = {}
    for name, prec, iters in (("fp64", 0, 12000), ("fp32", 1, 700000)):
        rates = []
        for _ in range(3):
            r = C.c_double(0.0)
            st = f(prec, blocks, threads, iters, C.c_void_p(out.data_ptr()),
                   C.byref(r), C.c_void_p(torch.cuda.current_stream().cuda_stream))
            if st != 0:
                raise RuntimeError("FMA probe failed (%d)" % st)
            rates.append(r.value)
        res[name] = {"tflops": max(rates) / 1e12, "runs_tflops": [x / 1e12 for x in rates]}
        _ALU[name] = max(rates)
    res["method"] = ("libcqprobe cq_probe_fma_rate: %d blocks x %d threads, 8 independent FMA chains per thread; "
                     "best of 3 timed launches" % (blocks, threads))
    res["nominal_fp64_tflops"] = FP64_PEAK_NOMINAL / 1e12
    return res


def alu_peak(name):
    """(peak FLOP/s, source) of the FP64 or FP32 pipe: the probe's figure from this run, else the
    nominal FP64 rate / a previous probe figure for FP32."""
    if name in _ALU:
        return _ALU[name], "FMA-rate probe in this run (libcqprobe, peaks.%s)" % name
    if name == "fp64":
        return FP64_PEAK_NOMINAL, "nominal FP64 rate (2 DFMA / clock / SM x 152 SMs x 2.07 GHz)"
    return FP32_PEAK_PROBE, "FMA-rate probe figure of an earlier run"


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

    def cproblem(q, prec=0):
        return fc.problem(q.alpha1, q.alpha2, q.m, q.T, q.N, q.dim, q.M, q.scheme, q.form, q.np1, q.np2, q.ns,
                          prec=prec, flags=flags)

    g0 = torch.tensor(G0, dtype=torch.float64, device=dev)
    gN = torch.empty_like(g0)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MiB > 2x L2
    fc.cq_timing_enable(True)

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(q, K, W, prec=0, accept=()):
        cp = cproblem(q, prec)
        ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), dev)
        for _ in range(W):
            fc.fp2s_solve(cp, g0, gN, ws)
        st = fc.fp2s_status(cp, ws)
        if st not in (fc.CQ_OK,) + tuple(accept):
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
        peaks = fma_peaks(torch, dev) if rank == 0 else None
        steps, mains, launches, st_fast = timed(p, K, W)
        gN_fast = gN.cpu().numpy()
        pd = p.replace(form=ci.DIRECT)
        Kd, Wd = max(1, min(K, 4)), max(1, min(W, 1))
        d_steps, d_mains, d_launches, st_dir = timed(pd, Kd, Wd)
        # the direct form in double-float: the (1,1) mode's growth (e^1096) leaves the FP32
        # exponent range, so its run ends non-finite; the timing does not depend on the values
        dd_steps, dd_mains, dd_launches, st_ddf = timed(pd, Kd, Wd, fc.CQ_DF64, accept=(fc.CQ_ENONFINITE,))
        gN_dir = gN.cpu().numpy()
        # the same fast solve in the double-float form (FP64-class accuracy on the FP32 pipe)
        df_steps, df_mains, df_launches, st_df = timed(p, K, W, fc.CQ_DF64)
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
    # the same workload on its sine coefficients (fp2s_solve_modes, no transform): the modal
    # result for the parity check against the oracle
    gm_fast = gm_dir = None
    if rank == 0:
        from oracle import spatial as OSP
        g0m = torch.tensor(OSP.to_modal(G0, p.M, p.dim), dtype=torch.float64, device=dev)
        gm_fast, gm_dir = (_modal_solve(fc, torch, dev, cproblem(q), g0m) for q in (p, p.replace(form=ci.DIRECT)))
        gm_df = _modal_solve(fc, torch, dev, cproblem(p, fc.CQ_DF64), g0m)
        gm_ddf = _modal_solve(fc, torch, dev, cproblem(p.replace(form=ci.DIRECT), fc.CQ_DF64), g0m, lo=p.M + 1)
        del g0m

    ms = statistics.mean(steps)
    ms_main = statistics.mean(mains)
    ms_dir = statistics.mean(d_steps)
    ms_e2e = statistics.mean(e2e)
    ms_df = statistics.mean(df_steps)
    if dist is not None:
        t = torch.tensor([ms, ms_dir, ms_e2e, ms_df], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_dir, ms_e2e, ms_df = t.tolist()
    units = p.ndof * p.N
    value = world * units / (ms * 1e-3)
    if rank != 0:
        return None

    # roofline of the dominant kernel (fused fast solve): FP64-pipe bound
    hist_flops_per_dof_step = 4 * (p.np1 + p.np2) + 2 * (p.ns - 1)
    flops_per_launch = hist_flops_per_dof_step * units
    achieved = flops_per_launch / (ms_main * 1e-3)
    pk, pk_src = alu_peak("fp64")
    roofline = {"kernel": "k_fp2s_fast", "bound": "alu", "unit": "TFLOP/s",
                "achieved": achieved / 1e12, "peak": pk / 1e12, "frac": achieved / pk, "peak_source": pk_src,
                "frac_of_nominal_fp64": achieved / FP64_PEAK_NOMINAL,
                "traffic": None, "algorithmic_flops_per_launch": flops_per_launch,
                "flops_per_dof_step": hist_flops_per_dof_step, "kernel_ms": ms_main,
                "kernel_share_of_step": ms_main / ms}
    traffic = _profiled_traffic("k_fp2s_fast_bdf2_2d_m255.md")
    if traffic is not None:
        roofline["traffic"] = traffic
        roofline["traffic_note"] = "ncu dram bytes of one full-size launch (the state stays on chip)"

    # oracle legs: bounded samples, which also give the errors of this run
    import numpy as np
    pd = p.replace(form=ci.DIRECT)
    sample, ref_fast, t_fast = oracle_sample(p, G0, args.cpu_modes, ci.SEED_BASE + 21)
    sample_d, ref_dir, t_dir = oracle_sample(pd, G0, max(4, args.cpu_modes // 16), ci.SEED_BASE + 22)
    cpu_fast = cpu_baseline(
        UNIT, 2 * len(sample) * p.N, t_fast, "oracle fast SBD scheme, %d seeded sine modes x all %d steps"
        % (len(sample), p.N), mode_jobs(p, G0, args.cpu_modes, [ci.SEED_BASE + 100 + k for k in range(_ncpu())]),
        _ncpu() * 2 * args.cpu_modes * p.N, "oracle fast SBD scheme, %d seeded sine modes x all %d steps per job"
        % (args.cpu_modes, p.N))
    nd = max(4, args.cpu_modes // 16)
    cpu_dir = cpu_baseline(
        UNIT, 2 * len(sample_d) * p.N, t_dir, "oracle direct SBD scheme, %d seeded modes x %d steps"
        % (len(sample_d), p.N), mode_jobs(pd, G0, nd, [ci.SEED_BASE + 120 + k for k in range(_ncpu())]),
        _ncpu() * 2 * nd * p.N, "oracle direct SBD scheme, %d seeded modes x %d steps per job" % (nd, p.N))
    error = {"fast": modal_parity(p, G0, gm_fast, sample, ref_fast),
             "direct": modal_parity(pd, G0, gm_dir, sample_d, ref_dir)}
    error["fast_df64"] = modal_parity(p, G0, gm_df, sample, ref_fast)
    sc = np.max(np.abs(gm_dir))
    error["fast_vs_direct_rel_l2"] = float(np.linalg.norm((gm_fast - gm_dir) / sc) / np.linalg.norm(gm_dir / sc))
    error["status"] = fc.strerror(st_fast)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; see config)", "config": workload_config(p),
        "roofline": roofline,
        "cpu_baseline": cpu_fast,
        "e2e": {"value": world * units / (ms_e2e * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(G0.size * 8), "d2h_bytes_per_step": int(G0.size * 8),
                "ms_per_step": ms_e2e},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "device": torch.cuda.get_device_name(),
    }
    # secondary legs; the most informative ones last, where a truncated log keeps them
    if paper is not None:
        out["paper_runs"] = {"note": "the paper's CPU times are on unstated hardware: context only", **paper}
    if small is not None:
        out["small_1d"] = small
    if stream is not None:
        out["fast_history_stream"] = stream
    kms_dir = statistics.mean(d_mains)
    flops_dir = 2.0 * 2 * (p.ndof // 2) * p.N * (p.N - 1) / 2        # one FMA per history term
    pk64, pk64_src = alu_peak("fp64")
    out["direct"] = {"value": world * units / (ms_dir * 1e-3), "unit": UNIT, "ms_per_step": ms_dir, "steps": Kd,
                     "warmup": Wd, "kernel": "k_fp2s_direct<8>", "kernel_ms": kms_dir,
                     "gpu_launches": int(d_launches), "status": fc.strerror(st_dir), "cpu_baseline": cpu_dir,
                     "roofline": {"kernel": "k_fp2s_direct<8>", "bound": "alu", "unit": "TFLOP/s",
                                  "achieved": flops_dir / (kms_dir * 1e-3) / 1e12, "peak": pk64 / 1e12,
                                  "frac": flops_dir / (kms_dir * 1e-3) / pk64, "peak_source": pk64_src,
                                  "traffic": _recorded_traffic("k_fp2s_direct"),
                                  "algorithmic_flops_per_launch": flops_dir,
                                  "flops_definition": "2 flops per history term, 2 states x nmodes x N (N - 1) / 2 "
                                                      "terms"}}
    ms_ddf = statistics.mean(dd_steps)
    kms_ddf = statistics.mean(dd_mains)
    ops_ddf = 12.0 * 2 * (p.ndof // 2) * p.N * (p.N - 1) / 2          # double-float history terms
    dec = np.array([k for k in sample_d if k > p.M])
    ref_dec = ref_dir[:, np.isin(sample_d, dec)]
    err_ddf = []
    for s_ in range(2):
        r_, g_ = ref_dec[s_], gm_ddf[s_, dec]
        sc = np.max(np.abs(r_))
        err_ddf.append(float(np.linalg.norm((g_ - r_) / sc) / np.linalg.norm(r_ / sc)))
    out["direct"]["df64"] = {
        "value": world * units / (ms_ddf * 1e-3), "unit": UNIT, "ms_per_step": ms_ddf,
        "kernel": "k_fp2s_direct_df<8>", "kernel_ms": kms_ddf, "speedup_vs_fp64_direct": ms_dir / ms_ddf,
        "gpu_launches": int(dd_launches), "status": fc.strerror(st_ddf),
        "status_note": "the (1,1) mode grows like e^(1096 t), past the FP32 exponent range the double-float "
                       "form keeps each mode in; the other modes are unaffected",
        "rel_l2_per_state_vs_oracle_decaying_modes": err_ddf, "decaying_modes_compared": int(len(dec)),
        "roofline": {"kernel": "k_fp2s_direct_df<8>", "bound": "alu", "unit": "T FP32-op/s",
                     "achieved": ops_ddf / (kms_ddf * 1e-3) / 1e12, "peak": alu_peak("fp32")[0] / 2e12,
                     "frac": ops_ddf / (kms_ddf * 1e-3) / (alu_peak("fp32")[0] / 2),
                     "fp32_ops_per_launch": ops_ddf,
                     "ops_definition": "12 FP32 operations per double-float history term, 2 states x nmodes x "
                                       "N (N - 1) / 2 terms"}}
    out["df64"] = df64_report(p, units, world, ms_df, statistics.mean(df_mains), ms, df_launches,
                              fc.strerror(st_df), error["fast_df64"], K, W)
    if peaks is not None:
        out["peaks"] = peaks
    if prec_leg is not None:
        out["precision"] = precision_report(prec_leg, 128)
    if grad is not None:
        out["gradient"] = grad
    if batch is not None:
        out["batch"] = batch
    out["error"] = error
    out["summary"] = summary(out)
    _close_pool()
    return out


def df64_fp32_ops_per_dof_step(p):
    """FP32-pipe operations of the double-float fast solve per DOF and step: per node 15 (update
    Y = r Y + G: TwoProduct with an FMA and TwoSum) or 23 (the slowest quarter of the node slots:
    Y = Y - u Y + G, two TwoSums) plus 12 (adding c Y to the sum), and 12 per window term."""
    npt = p.np1 + p.np2
    NP = next(b for b in (16, 32, 48, 64, 80) if npt <= b)
    ku = NP // 4
    return 27 * (NP - ku) + 35 * ku + 12 * (p.ns - 1)


def df64_report(p, units, world, ms, ms_main, ms_fp64, launches, status, error, K, W):
    """The headline workload in the double-float form (CQ_DF64): FP64-class accuracy from pairs
    of FP32 numbers on the FP32 pipe, the 2x2 step in FP64."""
    ops = df64_fp32_ops_per_dof_step(p)
    achieved = ops * units / (ms_main * 1e-3)
    pk, pk_src = alu_peak("fp32")
    flops64 = (4 * (p.np1 + p.np2) + 2 * (p.ns - 1)) * units
    return {
        "value": world * units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": K, "warmup": W,
        "speedup_vs_fp64_form": ms_fp64 / ms, "gpu_launches": int(launches), "status": status,
        "precision": "double-float (hi + lo FP32 pairs) node states, tables and history sums; FP64 2x2 step",
        "roofline": {"kernel": "k_fp2s_fast_df<80, SBD, 17>", "bound": "alu", "unit": "T FP32-op/s",
                     "achieved": achieved / 1e12, "peak": pk / 2e12, "frac": achieved / (pk / 2),
                     "peak_source": pk_src + " / 2 (one FMA = 2 flops = 1 FP32-pipe operation)",
                     "fp32_ops_per_dof_step": ops, "kernel_ms": ms_main,
                     "traffic": _recorded_traffic("k_fp2s_fast_df"),
                     "fp64_equivalent_tflops": flops64 / (ms_main * 1e-3) / 1e12},
        "error_vs_oracle": error,
        "cpu_baseline": "the headline's (the same oracle fast scheme)",
    }


def _modal_solve(fc, torch, dev, cp, g0m, lo=0):
    """The modal G^N of the modes lo .. nmodes - 1 through fp2s_solve_modes (numpy [2][nmodes];
    the columns before lo are NaN)."""
    import numpy as np
    nm = g0m.shape[1]
    src = g0m[:, lo:].contiguous()
    gN = torch.empty_like(src)
    ws = fc.workspace(fc.fp2s_solve_modes(cp, lo, nm, src, gN, None), dev)
    fc.fp2s_solve_modes(cp, lo, nm, src, gN, ws)
    out = np.full((2, nm), np.nan)
    out[:, lo:] = gN.cpu().numpy()
    del ws
    return out


def modal_parity(p, G0, gm, sample, ref):
    """GPU modal G^N against the oracle on sampled modes: relative L2 per state over the decaying
    modes; each growing mode's relative error beside its one-ulp conditioning (the change of the
    oracle's g^N when lambda_k, a or T moves by one unit in the last place)."""
    import numpy as np
    import cq_inputs as ci
    from oracle import scheme as OS
    from oracle import spatial as OSP
    lam_all = OSP.mode_eigenvalues(p.M, p.dim)
    grow = np.array([ci.growth_rate(p.alpha1, p.alpha2, p.m, lam_all[k]) > 0.0 for k in sample])
    got = gm[:, sample]
    rel = []
    for s in range(2):
        r, g = ref[s][~grow], got[s][~grow]
        sc = np.max(np.abs(r))
        rel.append(float(np.linalg.norm((g - r) / sc) / np.linalg.norm(r / sc)))
    g0m = OSP.to_modal(G0, p.M, p.dim)
    growing = []
    one = 2.0 ** -52
    for j in np.nonzero(grow)[0]:
        k = sample[j]
        lam_k, g0_k = lam_all[[k]], g0m[:, [k]]
        r_k = ref[:, [j]]
        moved = [OS.solve_modal(p, lam_k * (1 + one), g0_k)[p.N],
                 OS.solve_modal(p, lam_k, g0_k, a=OS.coupling(p.m) * (1 + one))[p.N],
                 OS.solve_modal(p.replace(T=p.T * (1 + one)), lam_k, g0_k)[p.N]]
        kappa = max(float(np.max(np.abs(m - r_k)) / np.max(np.abs(r_k))) for m in moved)
        growing.append({"mode": int(k), "rel_err": float(np.max(np.abs(got[:, [j]] - r_k)) / np.max(np.abs(r_k))),
                        "one_ulp_conditioning": kappa})
    return {"rel_l2_per_state_decaying_modes": rel, "decaying_modes": int((~grow).sum()),
            "growing_modes": growing,
            "method": "fp2s_solve_modes over all modes (the fused kernel, no transforms) against the oracle's "
                      "per-mode FP64 scheme on the sampled modes"}


def summary(out):
    """The headline figures of every leg in one place."""
    def g(d, *keys):
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d
    prec = out.get("precision", {})
    mixed = g(prec, "mixed_direct_solve") or {}
    cases = {("%s %s %s" % (c["scheme"], c["alpha"], c["contraction"])): c["rel_l2_err_vs_fp64_oracle"]
             for c in mixed.get("cases", [])}
    return {
        "headline": {"value": out["value"], "ms_per_step": out["ms_per_step"], "e2e": g(out, "e2e", "value"),
                     "roofline_frac": g(out, "roofline", "frac"), "roofline_peak_source": g(out, "roofline",
                                                                                            "peak_source")},
        "df64_fast_solve": {"value": g(out, "df64", "value"), "ms": g(out, "df64", "ms_per_step"),
                            "speedup_vs_fp64_form": g(out, "df64", "speedup_vs_fp64_form"),
                            "frac_fp32_pipe": g(out, "df64", "roofline", "frac"),
                            "rel_l2_per_state": g(out, "error", "fast_df64", "rel_l2_per_state_decaying_modes")},
        "direct_df64": {"ms": g(out, "direct", "df64", "ms_per_step"),
                        "speedup_vs_fp64_direct": g(out, "direct", "df64", "speedup_vs_fp64_direct"),
                        "rel_l2_per_state_decaying_modes": g(out, "direct", "df64",
                                                             "rel_l2_per_state_vs_oracle_decaying_modes")},
        "fp64_parity": {"fast": g(out, "error", "fast", "rel_l2_per_state_decaying_modes"),
                        "direct": g(out, "error", "direct", "rel_l2_per_state_decaying_modes"),
                        "fast_vs_direct_rel_l2": g(out, "error", "fast_vs_direct_rel_l2")},
        "fp32_fast_solve": {"ms": g(prec, "fp32_fast_solve", "ms_per_step"),
                            "rel_err": g(prec, "fp32_fast_solve", "error_vs_fp64_oracle_rel_l2_sampled_modes"),
                            "frac": g(prec, "fp32_fast_solve", "roofline", "frac")},
        "mixed_direct_solve": {"ms": mixed.get("ms_per_solve"), "contraction_frac": g(mixed, "roofline", "frac"),
                               "rel_l2_per_state": cases},
        "tensor_core_history": {"bf16x3_frac": g(prec, "tensor_core_direct_history", "roofline", "frac"),
                                "tf32x3_frac": g(prec, "tensor_core_direct_history_tf32x3", "roofline", "frac")},
        "batch": {"value": g(out, "batch", "value"), "graph_replay_value": g(out, "batch", "graph_replay", "value"),
                  "df64_value": g(out, "batch", "df64", "value"),
                  "df64_max_diff_vs_fp64": g(out, "batch", "df64", "max_abs_diff_vs_fp64_batch_rel_to_instance_max"),
                  "launch_shape": g(out, "batch", "launch_shape")},
        "gradient": {"ms": g(out, "gradient", "ms_per_gradient"),
                     "rel_err_vs_central_differences": g(out, "gradient", "rel_err_vs_central_differences"),
                     "df64": {"ms": g(out, "gradient", "df64", "ms_per_gradient"),
                              "rel_err_vs_central_differences": g(out, "gradient", "df64",
                                                                  "rel_err_vs_central_differences"),
                              "rel_err_vs_fp64_gradient": g(out, "gradient", "df64", "rel_err_vs_fp64_gradient")},
                     "fast": {"ms": g(out, "gradient", "fast", "ms_per_gradient"),
                              "df64_ms": g(out, "gradient", "fast", "df64", "ms_per_gradient"),
                              "rel_err_vs_central_differences": g(out, "gradient", "fast",
                                                                  "rel_err_vs_central_differences"),
                              "frac_fp64": g(out, "gradient", "fast", "roofline", "frac")},
                     "mixed": [{"precision": m.get("precision", "")[:6], "ms": m.get("ms_per_gradient"),
                                "rel_err_vs_fp64_gradient": m.get("rel_err_vs_fp64_gradient")}
                               for m in g(out, "gradient", "mixed_precision") or []]},
        "cpu_baselines_all_cores": {k: g(v, "cpu_baseline", "value") for k, v in (
            ("headline", out), ("direct", out.get("direct")), ("batch", out.get("batch")),
            ("gradient", out.get("gradient")), ("small_1d", out.get("small_1d")),
            ("fp32_fast", prec.get("fp32_fast_solve")), ("mixed", mixed),
            ("tensor_core_history", prec.get("tensor_core_direct_history")))},
        "cpu": cpu_info(),
    }


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


# Source files whose text a recorded traffic figure depends on, per kernel.
TRAFFIC_SOURCES = {
    "k_fp2s_fast_df": ("fastdf.cu", "fastdf.cuh", "fp2s_core.cuh", "common.cuh"),
    "k_fp2s_fast_f32": ("fp2s.cu", "fp2s_core.cuh", "common.cuh"),
    "k_fp2s_direct": ("fp2s.cu", "fp2s_core.cuh", "common.cuh"),
}
TRAFFIC_PROFILE = "dram_traffic_fused_solves_full_size.md"


def _files_hash(names):
    import hashlib
    h = hashlib.sha256()
    for f in names:
        with open(os.path.join(ROOT, "paper_1901_05128_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _recorded_traffic(kernel):
    """DRAM bytes per full-size launch of `kernel` recorded in profiles/ (one-pass ncu capture), if
    it was taken on the current text of the kernel's source files; else None."""
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", TRAFFIC_PROFILE)).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch\[%s\]: (\d+) \(source hash ([0-9a-f]+)\)" % re.escape(kernel), txt)
    if not m or m.group(2) != _files_hash(TRAFFIC_SOURCES[kernel]):
        return None
    return int(m.group(1))


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
    """The reference arm: the oracle (the paper's scheme in plain FP64 numpy) on the host's cores,
    one spawned process per core, each step a bounded sample of the workload (every process
    solves args.ref_modes seeded sine modes over all N steps)."""
    if rank != 0:
        return None
    import cq_inputs as ci
    p, G0 = ci.workload(WORKLOAD)
    G0 = G0 * SCALE
    n, ncpu = args.ref_modes, _ncpu()
    pool = _oracle_pool()
    short = p.replace(N=64, T=p.T * 64 / p.N)
    for w in range(args.warmup):
        pool.map(_oracle_job, mode_jobs(short, G0, n, [ci.SEED_BASE + 300 + 100 * w + k for k in range(ncpu)]),
                 chunksize=1)
    times = []
    for step in range(args.steps):
        jobs = mode_jobs(p, G0, n, [ci.SEED_BASE + 1000 + 100 * step + k for k in range(ncpu)])
        t = time.perf_counter()
        pool.map(_oracle_job, jobs, chunksize=1)
        times.append(time.perf_counter() - t)
    _close_pool()
    ms = 1e3 * statistics.mean(times)
    value = ncpu * 2 * n * p.N / (ms * 1e-3)
    info = cpu_info()
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; see config)",
            "config": workload_config(p),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncpu, "kind": "oracle", "cpu_model": info["model"],
                             "sample": "each step: %d spawned processes (one per core), each solving the oracle's "
                                       "fast SBD scheme on %d seeded sine modes x all %d steps (warm-up steps use "
                                       "N=64)" % (ncpu, n, p.N)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-modes", type=int, default=2048, help="sine modes of the oracle's timed sample (per job)")
    ap.add_argument("--ref-modes", type=int, default=2048,
                    help="sine modes per process and step of the reference arm")
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
