"""The convergence studies of Sec. 5 (Tables 1-5) run with the GPU solver.

    python -m paper_1901_05128_gb300.tables [table1 ... table5]

Every table solves the 1D two-state system on (0,1) with the initial data (a)
G1 = x(1-x), G2 = sin x or (b) G1 = (1-x) chi_(1/2,1), G2 = x chi_(0,1/2) (Sec. 5),
once with the plain scheme (BE Eq. 4.1 / SBD Eq. 4.7) and once with its fast form
(Eq. 4.3 / Eq. 4.8), and reports E_i = ||G_i^N - G_i,ref||_L2 against a reference
solution of the plain scheme with a smaller step, the rates log2(E(tau)/E(tau/2)),
and the GPU time of each solve.

Choices the paper leaves open (the numbers of quadrature points of the fast forms,
the reference step of Tables 1-2) are fixed here: Tables 1-2 take tau_ref = 1/6400
(the printed rates need it; the text says 1/3200), the fast BE form N_p = 96, the
fast SBD form N_p1 = 16, N_p2 = 64, N_s = 17 for T = 1 and N_p2 = 240 for the
N = 20000 steps of Table 5: a fixed Gauss-Jacobi rule loses the algebraic tail of
the weights beyond i ~ N_p2^2 (sum_i |eps_i| is 8 % of sum_i |d_i| with 64 points at
tau = 1/2000, N = 20000, and 1e-6 with 240).
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import cq_inputs as ci  # noqa: E402

# a = (1 - m) / (2m - 1): a = 2 <-> m = 0.6, a = -1 <-> m = 0
EXPERIMENTS = {
    "table1": dict(data="a", scheme=ci.BE, m=0.6, M=255, T=1.0, inv_tau=[100, 200, 400, 800, 1600],
                   ref_inv_tau=6400, alphas=[(0.3, 0.6), (0.4, 0.7)], fast=(96, 0, 2)),
    "table2": dict(data="b", scheme=ci.BE, m=0.6, M=255, T=1.0, inv_tau=[100, 200, 400, 800, 1600],
                   ref_inv_tau=6400, alphas=[(0.3, 0.7), (0.4, 0.6)], fast=(96, 0, 2)),
    "table3": dict(data="a", scheme=ci.BDF2, m=0.0, M=1023, T=1.0, inv_tau=[20, 40, 80, 160, 320],
                   ref_inv_tau=640, alphas=[(0.3, 0.4), (0.7, 0.8)], fast=(16, 64, 17)),
    "table4": dict(data="b", scheme=ci.BDF2, m=0.0, M=1023, T=1.0, inv_tau=[20, 40, 80, 160, 320],
                   ref_inv_tau=640, alphas=[(0.2, 0.4), (0.6, 0.8)], fast=(16, 64, 17)),
    "table5": dict(data="b", scheme=ci.BDF2, m=0.0, M=1023, T=10.0, inv_tau=[2000],
                   ref_inv_tau=4000, alphas=[(0.3, 0.8), (0.4, 0.7), (0.5, 0.6)], fast=(16, 240, 17)),
}


def initial_data(data: str, M: int) -> np.ndarray:
    return ci.g0_smooth_1d(M) if data == "a" else ci.g0_nonsmooth_1d(M)


def _solve(fc, torch, q: "ci.Problem", g0):
    cp = fc.problem(q.alpha1, q.alpha2, q.m, q.T, q.N, q.dim, q.M, q.scheme, q.form, q.np1, q.np2, q.ns)
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None), g0.device)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fc.fp2s_solve(cp, g0, gN, ws)
    e1.record()
    e1.synchronize()
    return gN.cpu().numpy(), e0.elapsed_time(e1) / 1e3


def run(name: str, fc=None, torch=None) -> dict:
    """Errors [alpha][form][step][component], rates and GPU seconds of one table."""
    if fc is None:
        import torch as _torch

        from . import build, load
        build()
        fc, torch = load(), _torch
    ex = EXPERIMENTS[name]
    M, T = ex["M"], ex["T"]
    h = 1.0 / (M + 1)
    g0 = torch.tensor(initial_data(ex["data"], M), dtype=torch.float64, device="cuda")
    out = {"name": name, "inv_tau": ex["inv_tau"], "rows": []}
    for a1, a2 in ex["alphas"]:
        base = ci.Problem(a1, a2, ex["m"], T, int(round(ex["ref_inv_tau"] * T)), 1, M, ex["scheme"], ci.DIRECT)
        ref, _ = _solve(fc, torch, base, g0)
        row = {"alpha": (a1, a2), "ref_norm": np.sqrt(h * np.sum(ref ** 2, axis=1))}
        for form in (ci.DIRECT, ci.FAST):
            errs, secs = [], []
            for it in ex["inv_tau"]:
                np1, np2, ns = ex["fast"]
                q = base.replace(N=int(round(it * T)), form=form, np1=np1, np2=np2, ns=ns)
                G, t = _solve(fc, torch, q, g0)
                errs.append(np.sqrt(h * np.sum((G - ref) ** 2, axis=1)))
                secs.append(t)
            E = np.array(errs)
            rates = np.log2(E[:-1] / E[1:]) if len(E) > 1 else np.zeros((0, 2))
            row["direct" if form == ci.DIRECT else "fast"] = {"E": E, "rates": rates, "gpu_s": secs}
        out["rows"].append(row)
    return out


def _print(res: dict):
    names = {ci.BE: ("BE", "FBE"), ci.BDF2: ("SBD", "FSBD")}[EXPERIMENTS[res["name"]]["scheme"]]
    print("%s  1/tau: %s" % (res["name"], " ".join("%10d" % v for v in res["inv_tau"])))
    for row in res["rows"]:
        for form, label in zip(("direct", "fast"), names):
            r = row[form]
            for c in range(2):
                vals = " ".join("%10.3e" % v for v in r["E"][:, c])
                print("(%.1f,%.1f) %-4s E%d   %s" % (row["alpha"][0], row["alpha"][1], label, c + 1, vals))
                if len(r["rates"]):
                    print("%16s rate %s" % ("", " " * 11 + " ".join("%10.4f" % v for v in r["rates"][:, c])))
            print("%16s GPU s %s" % ("", " ".join("%10.4f" % v for v in r["gpu_s"])))
        print("(%.1f,%.1f) |G_ref| %10.3e %10.3e" % (row["alpha"][0], row["alpha"][1], *row["ref_norm"]))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("tables", nargs="*", default=sorted(EXPERIMENTS))
    a = ap.parse_args(argv)
    for name in a.tables:
        _print(run(name))


if __name__ == "__main__":
    main()
