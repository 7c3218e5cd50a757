"""Command-line runner: solve one named synthetic workload on the GPU.

    python -m paper_1901_05128_gb300.run --workload bdf2_2d_m255 --form fast --repeat 2

Prints one line per solve with its wall time and the library status. Useful
for profiling a single configuration (e.g. under ncu).
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
    ap.add_argument("--prec", choices=["f64", "f32"], default="f64")
    a = ap.parse_args(argv)

    import torch

    import cq_inputs as ci
    from . import build, load

    build()
    fc = load()
    p, G0 = ci.workload(a.workload)
    if a.form:
        p = p.replace(form=ci.FAST if a.form == "fast" else ci.DIRECT)
    if a.scheme:
        p = p.replace(scheme=ci.BE if a.scheme == "be" else ci.BDF2)
    if a.N:
        p = p.replace(N=a.N, T=p.T * a.N / p.N)
    cp = fc.problem(p.alpha1, p.alpha2, p.m, p.T, p.N, p.dim, p.M, p.scheme, p.form, p.np1, p.np2, p.ns,
                    prec=fc.CQ_F32 if a.prec == "f32" else fc.CQ_F64)
    g0 = torch.tensor(G0 * 2.0 ** a.scale_exp, dtype=torch.float64, device="cuda")
    gN = torch.empty_like(g0)
    ws = fc.workspace(fc.fp2s_solve(cp, g0, gN, None))
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        st = fc.fp2s_solve(cp, g0, gN, ws, check=False)
        torch.cuda.synchronize()
        print("solve %d: %.3f s status=%s" % (r, time.perf_counter() - t, fc.strerror(st)))


if __name__ == "__main__":
    main()
