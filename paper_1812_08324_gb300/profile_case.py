"""Run one piece of the hot path on a chosen size, for profilers.

    python -m paper_1812_08324_gb300.profile_case --n 32768 --what solve --reps 3

Builds the H-matrix of the 1D Levy generator workload (drift 0.3, sigma 0.2,
alpha-stable alpha = 1.5 truncated to |y| <= 2, leaf 256, ACA rank <= 32,
factor rank <= 16, dt = 1e-3) at N unknowns, factors I - dt/2 G, then runs
one warm-up and `reps` timed repetitions of the chosen operation:
  matvec   y = x + dt/2 G x (H-matvec)
  solve    z = (LU)^{-1} b (the persistent solve schedule; the factorisation
           is the first launch of the same executor kernel)
  cn_step  one Crank-Nicolson step (right-hand side H-matvec + solve)
and prints the mean time per repetition (CUDA events).
"""
from __future__ import annotations

import argparse
import json

from . import build, hmat, workloads as W


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--what", choices=["matvec", "solve", "cn_step"], default="solve")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    import torch

    build.build()
    hmat.load()
    prob = W.levy_1d(args.n)
    _, opts, dt, _, kind = W.WORKLOADS["levy_1d_n65536"]
    opts = dict(opts, lu_max_rank=16, lu_tol=1e-10, refine_max=0)
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    x = torch.tensor(W.initial_data(prob, kind), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)

    def op():
        if args.what == "matvec":
            H.matvec(x, alpha=1.0, beta=0.5 * dt, out=y)
        elif args.what == "solve":
            F.solve(x, out=y)
        else:
            hmat.cn_step(H, F, dt, x, out=y)

    op()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        op()
    e1.record()
    torch.cuda.synchronize()
    st = H.stats(F)
    print(json.dumps({"n": args.n, "what": args.what, "reps": args.reps,
                      "ms": e0.elapsed_time(e1) / max(args.reps, 1),
                      "h_bytes": st["h_bytes"], "lu_bytes": st["lu_bytes"]}))
    F.free()
    H.free()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
