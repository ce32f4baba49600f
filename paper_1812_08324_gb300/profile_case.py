"""Run one piece of the hot path on a chosen size, for profilers.

    python -m paper_1812_08324_gb300.profile_case --n 32768 --what solve --reps 3

Builds the H-matrix of the 1D Levy generator workload (drift 0.3, sigma 0.2,
alpha-stable alpha = 1.5 truncated to |y| <= 2, leaf 256, ACA rank <= 32,
factor rank <= 16, dt = 1e-3) at N unknowns (or, with --workload, of another
named workload: a 2D fractional Laplacian on a grid of side sqrt(N)), factors
I - dt/2 G, then runs
one warm-up and `reps` timed repetitions of the chosen operation:
  matvec   y = x + dt/2 G x (H-matvec: vt_kernel, vt_reduce_kernel, rows_kernel)
  solve    z = (LU)^{-1} b (1D: the hierarchical inverses' products, hinv_t_kernel
           and hinv_r_kernel per factor)
  cn_step  one Crank-Nicolson step (identity form: one pair of solves)
  factor   the H-LU of I - dt/2 G again (the executor's exec_kernel<0>
           launches; HM_PIPELINE=0 makes it one launch) and the hierarchical
           inverses' construction
and prints the mean time per repetition (CUDA events).  With --trace PREFIX
the timed repetitions run with the executor's per-task trace (HM_PHASE_TRACE,
HM_TRACE_FILE=PREFIX; read by ``python -m paper_1812_08324_gb300.trace_chain``)
and the trace files are gzip-compressed afterwards.
"""
from __future__ import annotations

import argparse
import gzip
import json
import os
import shutil

from . import build, hmat, workloads as W


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--workload", default="levy_1d_n65536",
                    help="named workload whose physics and options are used (1D Levy: N = --n; the 2D "
                         "fractional Laplacian workloads: grid side sqrt(--n))")
    ap.add_argument("--what", choices=["matvec", "solve", "cn_step", "factor"], default="solve")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--solve", choices=["auto", "hinv", "subst"], default="auto",
                    help="triangular solves: hierarchical inverses (1D default) or substitution")
    ap.add_argument("--trace", default=None, help="file prefix of the per-task trace of the timed repetitions")
    args = ap.parse_args()
    import torch

    build.build()
    hmat.load()
    prob, opts, dt, _, kind = W.WORKLOADS[args.workload]
    if prob["dim"] == 1:
        prob = W.levy_1d(args.n) if args.workload.startswith("levy_1d") else dict(prob)
    else:
        prob = W.frac_lap_2d(int(round(args.n ** 0.5)), prob["s"])
    opts = dict(opts, lu_max_rank=16, lu_tol=1e-10, refine_max=0, solve=args.solve)
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    x = torch.tensor(W.initial_data(prob, kind), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)

    def op():
        if args.what == "matvec":
            H.matvec(x, alpha=1.0, beta=0.5 * dt, out=y)
        elif args.what == "solve":
            F.solve(x, out=y)
        elif args.what == "factor":
            H.factor(-0.5 * dt).free()
        else:
            hmat.cn_step(H, F, dt, x, out=y)

    op()
    torch.cuda.synchronize()
    if args.trace:
        os.environ["HM_PHASE_TRACE"] = "1"
        os.environ["HM_TRACE_FILE"] = args.trace
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        op()
    e1.record()
    torch.cuda.synchronize()
    if args.trace:
        del os.environ["HM_PHASE_TRACE"], os.environ["HM_TRACE_FILE"]
        folder, stem = os.path.split(os.path.abspath(args.trace))
        for name in os.listdir(folder):
            if name.startswith(stem + ".") and name.endswith(".txt"):
                path = os.path.join(folder, name)
                with open(path, "rb") as a, gzip.open(path + ".gz", "wb") as b:
                    shutil.copyfileobj(a, b)
                os.remove(path)
    st = H.stats(F)
    print(json.dumps({"n": args.n, "what": args.what, "reps": args.reps,
                      "ms": e0.elapsed_time(e1) / max(args.reps, 1),
                      "h_bytes": st["h_bytes"], "lu_bytes": st["lu_bytes"]}))
    F.free()
    H.free()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
