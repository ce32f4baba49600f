"""Benchmark: Crank-Nicolson unknown-steps/s of the H-matrix Levy solver on GB300.

One bench *step* is one pass of the whole hot path over one synthetic input:
H-matrix assembly (tables, near field, ACA), H-LU of I - dt/2 G, and the full
CN run (each step one pair of triangular solves on v = u^n + u^{n+1}, plus
an H-matvec residual and a solve pair per FP64 refinement sweep) of the
1D full Levy generator workload (N = 65536, drift 0.3, sigma 0.2, alpha-stable
alpha = 1.5 truncated to |y| <= 2, leaf 256, ACA rank <= 32, 1000 CN steps,
dt = 1e-3).  The metric is unknown-steps/s = N * CN steps / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload levy_1d_n65536|levy_batch] [--batch-count C]

--workload lshape solves the variable-order fractional Poisson problem on
the L-shaped domain (H-LU-preconditioned Richardson; unknowns/s).
--workload serve serves a seeded Poisson request stream (continuous batching,
150 GB admission budget) and adds p50/p99 latency to the line.
--workload levy_batch measures the batched workload instead: 512 independent
1D Levy solves (splitmix64 seed 0: N = round(2^U(10,15)), alpha, drift,
sigma), leaf sizes from the autotuner, 500 CN steps each at dt = 1/500; one
step = build all H-matrices + one batched H-LU launch + the batched CN run.

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
replica (the solve does not shard); value = total unknown-steps / max time.
The reference arm times the dense FP64 CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "levy_1d_n65536"
METRIC = "CN unknown-steps/s at <=1e-6 rel err vs FP64 (H-matrix build + H-LU + CN run)"
UNIT = "unknown-steps/s"

# stored dense-oracle solutions for the accuracy figure of a workload: the
# same physics, options, dt and step count on a smaller grid (written by the
# scripts beside them, which call only the oracle)
ORACLE_GOLDEN = {
    "levy_1d_n65536": {
        "file": "tests/golden/levy1d_n32768_dt1e-3.npz", "steps": 1000,
        "prob": ("levy_1d", (32768,)),
        "what": "dense FP64 oracle (assembly + dense LU + 1000 CN steps) at N=32768, same physics, options "
                "and steps (tests/golden/levy1d_n32768_dt1e-3.npz)"},
    "frac_lap_2d_256x256_s0.75": {
        "file": "tests/golden/frac2d_n128_s0.75_dt5e-3.npz", "steps": 200,
        "prob": ("frac_lap_2d", (128, 0.75)),
        "what": "dense FP64 oracle (assembly + dense LU + 200 CN steps) at side 128 (N=16384), same order, "
                "options and steps (tests/golden/frac2d_n128_s0.75_dt5e-3.npz)"},
}

def load_peaks() -> dict:
    """The measured peaks (HBM copy GB/s, cuBLAS bf16 TFLOP/s, clocks), or {}."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


DF_PEAK_SOURCE = "derived: 128 FP32 lanes x 152 SMs x max SM clock / 10 instructions per double-float FMA"


def df_alu_peak(clocks) -> float:
    """TFLOP/s (FP64-equivalent) of double-float FMAs on the FP32 pipes: 128
    FP32 lanes per SM x 152 SMs x the maximum SM clock, 10 FP32 instructions
    per double-float FMA, 2 flop per FMA."""
    sm_mhz = (clocks or {}).get("sm_max_mhz") or load_peaks().get("sm_max_mhz") or 2070.0
    return 2.0 * 128 * 152 * sm_mhz * 1e6 / 10.0 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cn-steps", type=int, default=None, help="override the workload's CN steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--refine", type=int, default=None,
                    help="refinement sweeps per CN step (default: 0 for FP64, 1 for the mixed precisions)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed_fp32", "mixed_bf16"],
                    help="storage of what the triangular solves read (the mixed modes refine in FP64)")
    ap.add_argument("--solve", default="auto", choices=["auto", "hinv", "subst"],
                    help="triangular solves: hierarchical inverses (1D default) or substitution")
    ap.add_argument("--cn-form", default="identity", choices=["identity", "literal"],
                    help="CN step as (I - dt/2 G) v = 2u^n, u^{n+1} = v - u^n (no H-matvec), or with the "
                         "H-matvec right-hand side as the scheme is written")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "frac_lap_2d_256x256_s0.75",
                                                             "frac_lap_2d_256x256_s0.3", "levy_batch", "serve",
                                                             "lshape"])
    ap.add_argument("--lshape-n", type=int, default=255, help="grid side of the L-shaped Poisson workload")
    ap.add_argument("--serve-count", type=int, default=200)
    ap.add_argument("--serve-sides", default="64,128", help="2D grid sides of the served stream")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--group-unknowns", type=int, default=2400000)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(ms_local: float, units_local: float, world: int, device: str = "cpu"):
    """Whole-job timing over replicas: the slowest rank's time per step and the
    units all ranks processed per second (every rank runs the same replica)."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_local / (ms * 1e-3)


def workload(refine=0, name=WORKLOAD, precision="fp64", solve="auto", cn_form="identity"):
    from paper_1812_08324_gb300 import workloads as W
    prob, opts, dt, steps, kind = W.WORKLOADS[name]
    # the factors' low-rank blocks are capped at rank 16 or at the ACA ranks
    # if larger (1D: ACA ranks <= 9; 2D at ACA 1e-8: <= 25)
    if refine is None:
        refine = 0 if precision == "fp64" else 1
    opts = dict(opts, lu_max_rank=16, lu_tol=1e-10, refine_max=refine, precision=precision, solve=solve,
                cn_form=cn_form)
    return prob, opts, dt, steps, kind


def cpu_sample_2d(name, budget_n=64):
    """The dense oracle on a bounded sample of a 2D workload: the same
    fractional Laplacian at n = 64 per axis (N = 4096), dense assembly, dense
    LU and the workload's CN steps; unknown-steps/s over the sample."""
    from oracle import levy_dense as O
    from paper_1812_08324_gb300 import workloads as W
    prob, _, dt, steps, kind = W.WORKLOADS[name]
    small = dict(prob, n=[budget_n, budget_n])  # the window L_W = 1 is still (n + 1) h
    t0 = time.perf_counter()
    G = O.generator_dense(small)
    O.cn_solve(G, W.initial_data(small, kind), dt, steps)
    t = time.perf_counter() - t0
    n = budget_n * budget_n
    return {"value": n * steps / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"dense oracle on the same 2D problem at {budget_n}x{budget_n}: assembly + LU + {steps} CN steps, {t:.2f} s"}


def cpu_sample(steps_override=None, n=8192, steps=20):
    """The dense oracle, as it stands, on a bounded sample of the workload:
    the same 1D Levy physics at N = 8192 (h = 2/8193): dense assembly, dense
    LU of I - dt/2 G and `steps` CN steps (identity form, one LU solve per
    step), each phase timed.  Reports the sample's own unknown-steps/s and,
    labelled as an extrapolation, the rate at the workload's size (N = 65536,
    1000 steps) with the phases scaled by their cost laws: assembly N^2, LU
    N^3, a step N^2 (the oracle itself cannot run there: its host LU stops
    at 2^32 matrix entries)."""
    from oracle import levy_dense as O
    from paper_1812_08324_gb300 import workloads as W
    prob = W.levy_1d(n)
    _, _, dt, full_steps, _ = W.WORKLOADS[WORKLOAD]
    cn = steps if steps_override is None else max(1, min(steps, steps_override))
    t0 = time.perf_counter()
    G = O.generator_dense(prob)
    t1 = time.perf_counter()
    u0 = W.gaussian_u0(prob, 50.0)
    t2 = time.perf_counter()
    O.cn_solve(G, u0, dt, 0, literal=False)   # assembly of M and its LU
    t3 = time.perf_counter()
    O.cn_solve(G, u0, dt, cn, literal=False)  # LU again + cn steps
    t4 = time.perf_counter()
    t_asm, t_lu = t1 - t0, t3 - t2
    t_step = max((t4 - t3) - t_lu, 0.0) / cn
    sample_s = t_asm + t_lu + cn * t_step
    sample_rate = n * cn / sample_s
    big, ratio = 65536, 65536 / n
    t_big = t_asm * ratio ** 2 + t_lu * ratio ** 3 + full_steps * t_step * ratio ** 2
    cores = os.cpu_count()
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        cores = max((i.get("num_threads", 1) for i in info), default=cores)
    except Exception:
        pass
    return {"value": big * full_steps / t_big, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"dense oracle on the same 1D Levy physics at N={n}: assembly {t_asm:.2f} s, LU {t_lu:.2f} s, "
                       f"{cn} CN steps at {t_step * 1e3:.1f} ms ({sample_rate:.3g} unknown-steps/s over the sample); "
                       f"value = extrapolation to N={big}, {full_steps} steps (assembly x{ratio ** 2:.0f}, "
                       f"LU x{ratio ** 3:.0f}, steps x{ratio ** 2:.0f}): {t_big:.0f} s"),
            "sample_value": sample_rate, "extrapolated": True}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_sample(args.cn_steps)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_sample(args.cn_steps)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    value = args.steps / sum(1.0 / v for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle sample N=8192, extrapolated)"},
            "cpu_baseline": dict(last, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """The batched workload (see the module docstring)."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1812_08324_gb300 import autotune, build, hmat, workloads as W
    build.build()
    hmat.load()
    batch = W.levy_batch(args.batch_count)
    dt = W.LEVY_BATCH_DT
    cn_steps = args.cn_steps or W.LEVY_BATCH_STEPS
    refine = args.refine if args.refine is not None else (0 if args.precision == "fp64" else 1)
    batch = [(p, dict(o, refine_max=refine, precision=args.precision, solve=args.solve, cn_form=args.cn_form))
             for p, o in batch]
    cfgs = autotune.tune_batch_configs(batch, dt, cn_steps, probe_steps=3)
    batch = [(p, dict(o, **c)) for (p, o), c in zip(batch, cfgs)]
    leafs = [c["leaf"] for c in cfgs]
    ns = [p["n"][0] for p, _ in batch]
    units = float(sum(ns)) * cn_steps
    u0_host = [torch.tensor(W.gaussian_u0(p, 50.0), dtype=torch.float64).pin_memory() for p, _ in batch]
    u0_dev = [u.to("cuda") for u in u0_host]
    us = [torch.empty_like(u) for u in u0_dev]
    stream = torch.cuda.current_stream()

    # consecutive groups of at most group_unknowns unknowns share the GPU at a
    # time (the factors of all 512 problems would not fit in HBM at once)
    groups, cur, tot = [], [], 0
    for i, n in enumerate(ns):
        if cur and tot + n > args.group_unknowns:
            groups.append(cur)
            cur, tot = [], 0
        cur.append(i)
        tot += n
    groups.append(cur)

    def step(srcs, keep_last=False):
        kept = None
        for gi, g in enumerate(groups):
            Hs = [hmat.HMatrix(*batch[i]) for i in g]
            Fs = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
            for i in g:
                us[i].copy_(srcs[i])
            hmat.cn_solve_batch(Hs, Fs, dt, cn_steps, [us[i] for i in g])
            if keep_last and gi == len(groups) - 1:
                kept = (Hs, Fs, g)
            else:
                release(Hs, Fs)
        return kept

    def release(Hs, Fs):
        for F in Fs:
            F.free()
        for H in Hs:
            H.free()

    for _ in range(args.warmup):
        step(u0_dev)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    l0 = hmat.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(args.steps):
        kept = step(u0_dev, keep_last=k == args.steps - 1)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = (hmat.launch_count() - l0) // max(1, args.steps)
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = sampler.stop()
    ms, value = aggregate(ms, units, world, "cuda")
    graphed = hmat.batch_graphed()

    # accuracy: a few members against their converged solves (the batch equals the single path bit for bit)
    errs = []
    for i in np.linspace(0, len(batch) - 1, 3).astype(int):
        p, o = batch[i]
        H3 = hmat.HMatrix(p, dict(o, refine_max=3))
        F3 = H3.factor(-0.5 * dt)
        ur = u0_dev[i].clone()
        hmat.cn_solve(H3, F3, dt, cn_steps, ur)
        errs.append(float(torch.linalg.norm(us[i] - ur) / torch.linalg.norm(ur)))
        F3.free()
        H3.free()
    # CN part alone on the last group and its bytes per step (roofline of the batched step)
    Hs, Fs, g = kept
    sts = [H.stats(F) for H, F in zip(Hs, Fs)]
    # per CN step: one pair of solves, plus one H-matvec per refinement sweep
    # (and one for the right-hand side in the literal form)
    n_mv = refine + (1 if args.cn_form == "literal" else 0)
    byts = float(sum(st["lu_bytes"] + n_mv * st["h_bytes"] for st in sts))
    gus = [u0_dev[i].clone() for i in g]
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    hmat.cn_solve_batch(Hs, Fs, dt, 20, gus)
    c1.record(stream)
    torch.cuda.synchronize()
    cn_ms = c0.elapsed_time(c1) / 20
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    gbs = byts / (cn_ms * 1e-3) / 1e9
    roofline = {"kernel": "batched CN step (inverse products of the 1D members, merged substitution schedule, "
                          "batched H-matvec per sweep; one CUDA graph)",
                "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                "peak_source": "hbm_gbs " + ("of measured" if peaks else "of fallback"),
                "algorithmic_bytes": byts, "ms": cn_ms}

    # end to end from pinned host memory
    release(Hs, Fs)
    outs = [torch.empty_like(u).pin_memory() for u in u0_host]
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    devs = [u.to("cuda", non_blocking=True) for u in u0_host]
    step(devs)
    for o, u in zip(outs, us):
        o.copy_(u, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - e0
    e2e = {"value": world * units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * sum(ns),
           "d2h_bytes_per_step": 8 * sum(ns)}
    line = {"metric": METRIC.replace("(H-matrix build + H-LU + CN run)", "(batched: build + H-LU + CN run)"),
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"levy_batch x{len(batch)} (splitmix64 seed 0)", "sum_N": int(sum(ns)),
                       "cn_steps": cn_steps, "dt": dt, "leafs": {str(l): leafs.count(l) for l in sorted(set(leafs))},
                       "tuned": {f"leaf {c['leaf']}, {c['solve']}" + (f" blocks {c['solve_block']}" if c.get("solve_block") else ""):
                                 sum(1 for d in cfgs if d == c) for c in [dict(t) for t in sorted({tuple(sorted(d.items())) for d in cfgs})]},
                       "groups": len(groups), "group_unknowns_max": args.group_unknowns,
                       "refine_sweeps": refine, "precision": args.precision, "solve": args.solve, "cn_form": args.cn_form,
                       "parallelism": f"replicas x{world}", "cuda_graph": graphed,
                       "l2": "working set (H + factors of all problems) exceeds L2; no flush needed"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "accuracy": {"rel_l2_vs_converged_fp64_solves_sampled": errs,
                         "reference": "three members, same H-matrix CN run with 3 FP64 refinement sweeps per step"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_lshape(args):
    """The variable-order fractional Poisson problem on the L-shaped domain
    (Sec. "Application: Variable-Order Fractional Poisson Equation"): n x n
    interior grid of [-1,1]^2 without the upper-right quadrant, s(x) = 0.9 -
    0.8 d(x), three Gaussian sources.  One step = build the operator
    (ACA 1e-10) and the preconditioner H-matrix (eps_1 = 1e-4), H-LU of the
    latter (eps_2 = 1e-10), and H-LU-preconditioned Richardson iteration to a
    relative residual of 1e-12.  Unit: unknowns solved per second."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1812_08324_gb300 import build, hmat, workloads as W
    build.build()
    hmat.load()
    n = args.lshape_n
    prob = W.lshape_poisson(n)
    o_op = W.default_opts(leaf=256, aca_tol=1e-10, max_rank=64, refine_max=0)
    o_pre = W.default_opts(leaf=256, aca_tol=1e-4, max_rank=64, lu_tol=1e-10, lu_max_rank=48, refine_max=0)
    f_host = torch.tensor(W.lshape_source(prob), dtype=torch.float64).pin_memory()
    f = f_host.to("cuda")
    stream = torch.cuda.current_stream()
    info = {}

    def step(rhs):
        Hop = hmat.HMatrix(prob, o_op)
        Hpre = hmat.HMatrix(prob, o_pre)
        F = Hpre.factor_shifted(0.0, 1.0)
        u, it, res = hmat.shifted_solve(Hop, F, rhs, tol=1e-12, maxit=100)
        info.update(iters=it, resid=res)
        return Hop, Hpre, F, u

    def release(*xs):
        for x in xs:
            x.free()

    for _ in range(args.warmup):
        Hop, Hpre, F, u = step(f)
        release(F, Hpre, Hop)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    l0 = hmat.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(args.steps):
        Hop, Hpre, F, u = step(f)
        if k < args.steps - 1:
            release(F, Hpre, Hop)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = (hmat.launch_count() - l0) // max(1, args.steps)
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = sampler.stop()
    N = Hop.n
    ms, value = aggregate(ms, float(N), world, "cuda")
    s_op, s_pre = Hop.stats(), Hpre.stats(F)
    # roofline of the dominant kernel: the H-LU executor (double-float GEMM tiles on the FP32 pipes)
    peak = df_alu_peak(clocks)
    tflops = 2.0 * s_pre["factor_fma"] / (s_pre["factor_ms"] * 1e-3) / 1e12 if s_pre["factor_ms"] > 0 else None
    roofline = {"kernel": "exec_kernel<0> (H-LU schedule of the preconditioner, double-float GEMM tiles)",
                "bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                "frac": tflops / peak if tflops else None, "traffic": None, "peak_source": DF_PEAK_SOURCE,
                "algorithmic_flops": 2.0 * s_pre["factor_fma"], "ms": s_pre["factor_ms"]}
    # accuracy: sampled rows of the exact generator are checked in the tests; here the
    # residual against the accurate operator and the iteration count
    u_host = u.cpu().numpy()
    release(F, Hpre, Hop)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    fd = f_host.to("cuda", non_blocking=True)
    Hop, Hpre, F, u = step(fd)
    out = torch.empty(N, dtype=torch.float64).pin_memory()
    out.copy_(u, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - e0
    release(F, Hpre, Hop)
    e2e = {"value": world * N / e2e_s, "unit": "unknowns/s", "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N}
    line = {"metric": "variable-order fractional Poisson unknowns/s (build + H-LU preconditioner + "
                      "preconditioned Richardson to 1e-12)",
            "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"lshape_poisson_n{n} (N={N}, s(x)=0.9-0.8d(x))", "operator_aca_tol": 1e-10,
                       "preconditioner_aca_tol": 1e-4, "lu_tol": 1e-10, "leaf": 256,
                       "iterations": info["iters"], "final_rel_residual": info["resid"],
                       "operator_max_rank": s_op["max_rank_seen"], "preconditioner_max_rank": s_pre["max_rank_seen"],
                       "factor_max_rank": s_pre["lu_max_rank_seen"], "parallelism": f"replicas x{world}",
                       "l2": "H-matrices and factors exceed L2; no flush needed"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "solution_norm": float(np.linalg.norm(u_host))}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import variable_order as V
        t0 = time.perf_counter()
        ns = 63
        V.poisson_solve(V.lshape_problem(ns))
        t = time.perf_counter() - t0
        nn = ns * ns - ((ns + 1) // 2) ** 2
        line["cpu_baseline"] = {"value": nn / t, "unit": "unknowns/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"dense assembly + dense LU solve at n={ns} (N={nn})"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """The served request stream: Poisson arrivals (rate 200/s, splitmix64
    seed 0), half 1D (N = round(2^U(10,16))) and half 2D fractional Laplacian
    requests, s ~ U(0.2,0.9), 100..1000 CN steps, 150 GB admission budget.
    One bench step serves the whole stream; value = unknown-steps/s over the
    stream's span; latency percentiles per request (arrival to result on the
    host)."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_1812_08324_gb300 import build, hmat, serve, workloads as W
    build.build()
    hmat.load()
    sides = tuple(int(x) for x in args.serve_sides.split(","))
    reqs = W.serve_stream(args.serve_count, seed=0, rate=200.0, sides_2d=sides)
    warm = W.serve_stream(6, seed=1, rate=200.0, log2_1d=(10.0, 12.0), sides_2d=(32,), steps=(20, 40))
    for _ in range(args.warmup):
        serve.Server(hbm_budget=150e9).run(warm)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    l0 = hmat.launch_count()
    summaries = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        srv = serve.Server(hbm_budget=150e9, tick_steps=20)
        res = srv.run(reqs)
        summaries.append(serve.summary(res))
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / args.steps
    clocks = sampler.stop()
    launches = (hmat.launch_count() - l0) // max(1, args.steps)
    last = summaries[-1]
    work = float(sum(r.n * r.steps for r in res))
    value = work / wall
    # a sample of results against the same requests solved alone with refinement
    errs = []
    for r, q in list(zip(res, reqs))[:: max(1, len(reqs) // 3)][:3]:
        H = hmat.HMatrix(q["problem"], dict(q["opts"], refine_max=3))
        F = H.factor(-0.5 * q["dt"])
        u = torch.tensor(q["u0"], dtype=torch.float64, device="cuda")
        hmat.cn_solve(H, F, q["dt"], q["steps"], u)
        ref = u.cpu().numpy()
        errs.append(float(np.linalg.norm(r.u - ref) / np.linalg.norm(ref)))
        F.free()
        H.free()
    ns1 = [r.n for r, q in zip(res, reqs) if q["problem"]["dim"] == 1]
    ns2 = [r.n for r, q in zip(res, reqs) if q["problem"]["dim"] == 2]
    line = {"metric": METRIC.replace("(H-matrix build + H-LU + CN run)", "(served stream: admission + build + H-LU + CN run)"),
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"serve_stream x{len(reqs)} (Poisson 200/s, splitmix64 seed 0)",
                       "requests_1d": len(ns1), "requests_2d": len(ns2), "sides_2d": list(sides),
                       "sum_N_steps": work, "hbm_budget_bytes": 150e9, "tick_steps": 20,
                       "peak_device_bytes": srv.peak_used, "batches_built": srv.batches_built,
                       "l2": "working set exceeds L2; no flush needed"},
            "latency": {"p50_s": last["p50_latency_s"], "p99_s": last["p99_latency_s"], "span_s": last["span_s"]},
            "clocks": clocks,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 8 * sum(r.n for r in res),
                    "d2h_bytes_per_step": 8 * sum(r.n for r in res),
                    "note": "the server run is end to end: host u0 in, host result out per request"},
            "gpu_launches": int(launches), "roofline": None,
            "accuracy": {"rel_l2_vs_alone_refined_sampled": errs}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample()
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "levy_batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "lshape":
        return run_lshape(args)
    import numpy as np
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1812_08324_gb300 import build, hmat
    build.build()
    hmat.load()
    from paper_1812_08324_gb300 import workloads as W

    name = args.workload
    prob, opts, dt, cn_steps, kind = workload(args.refine, name, args.precision, args.solve, args.cn_form)
    if args.cn_steps:
        cn_steps = args.cn_steps
    N = prob["n"][0] * (prob["n"][1] if prob["dim"] == 2 else 1)
    u0_host = torch.tensor(W.initial_data(prob, kind), dtype=torch.float64).pin_memory()
    u0 = u0_host.to("cuda")
    u = torch.empty_like(u0)
    stream = torch.cuda.current_stream()

    def step(dev_in, out):
        H = hmat.HMatrix(prob, opts)
        F = H.factor(-0.5 * dt)
        out.copy_(dev_in)
        hmat.cn_solve(H, F, dt, cn_steps, out)
        return H, F

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        H, F = step(u0, u)
    torch.cuda.synchronize()
    H.sync()
    st = H.stats(F)

    # ---- device-resident timed region
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = hmat.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        H, F = step(u0, u)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = (hmat.launch_count() - l0) // max(1, args.steps)
    ms = ev0.elapsed_time(ev1) / args.steps
    clocks = sampler.stop()
    H.sync()
    ms, value = aggregate(ms, N * cn_steps, world, "cuda")

    # ---- accuracy of the timed configuration: (1) the same CN run with three
    # FP64 refinement sweeps per step (solves converged to the FP64 H system);
    # (2) against the dense FP64 oracle: the same physics, options and steps
    # on the largest grid whose dense LU the host reaches, u stored by the
    # scripts under tests/golden (ORACLE_GOLDEN)
    assert torch.isfinite(u).all().item()
    u_ref = torch.empty_like(u0)
    Href = hmat.HMatrix(prob, dict(opts, refine_max=3, precision="fp64"))
    Fref = Href.factor(-0.5 * dt)
    u_ref.copy_(u0)
    hmat.cn_solve(Href, Fref, dt, cn_steps, u_ref)
    torch.cuda.synchronize()
    rel_err = float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref))
    Fref.free()
    Href.free()
    oracle_err, oracle_ref = None, None
    gold = ORACLE_GOLDEN.get(name)
    if gold is not None and cn_steps == gold["steps"] and os.path.exists(os.path.join(ROOT, gold["file"])):
        g = np.load(os.path.join(ROOT, gold["file"]))
        p_s = getattr(W, gold["prob"][0])(*gold["prob"][1])
        H_s = hmat.HMatrix(p_s, opts)
        F_s = H_s.factor(-0.5 * dt)
        u_s = torch.tensor(W.initial_data(p_s, kind), dtype=torch.float64, device="cuda")
        hmat.cn_solve(H_s, F_s, dt, cn_steps, u_s)
        got = u_s.cpu().numpy()
        want = g[f"u{cn_steps}"]
        oracle_err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        oracle_ref = gold["what"]
        F_s.free()
        H_s.free()

    # ---- end to end through the public API from pinned host memory
    out_host = torch.empty(N, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        dev = u0_host.to("cuda", non_blocking=True)
        H, F = step(dev, u)
        out_host.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - e0) / args.steps
    e2e = {"value": world * N * cn_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * N,
           "d2h_bytes_per_step": 8 * N}

    # ---- rooflines.  Per CN step: the H-matvec (three launches) and the two
    # triangular solves (hierarchical inverses: four launches; substitution:
    # one executor launch), timed with CUDA events on the launching stream;
    # per bench step: the H-LU executor (device time of its launches, CUDA
    # events inside the library).  The `roofline` object is the kernel with
    # the largest time per bench step.
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_src = "of measured" if peaks else "of fallback"
    x = torch.tensor(W.initial_data(prob, kind), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e_a.record(stream)
        for _ in range(reps):
            fn()
        e_b.record(stream)
        torch.cuda.synchronize()
        return e_a.elapsed_time(e_b) / reps

    mv_ms = timed(lambda: H.matvec(x, alpha=1.0, beta=0.5 * dt, out=y), 50)
    sv_ms = timed(lambda: F.solve(x, out=y), 50)
    mv_gbs = st["h_bytes"] / (mv_ms * 1e-3) / 1e9
    sv_gbs = st["lu_bytes"] / (sv_ms * 1e-3) / 1e9
    hinv = st["solve_mode"] == 2
    sweeps = opts["refine_max"]
    n_mv = cn_steps * (sweeps + (1 if opts["cn_form"] == "literal" else 0))
    n_sv = cn_steps * (1 + sweeps)
    mv_roof = {"kernel": "H-matvec (vt_kernel + vt_reduce + rows_kernel)", "bound": "hbm", "achieved": mv_gbs,
               "peak": hbm, "unit": "GB/s", "frac": mv_gbs / hbm, "traffic": None,
               "algorithmic_bytes": st["h_bytes"], "ms": mv_ms, "per_bench_step_ms": n_mv * mv_ms,
               "peak_source": f"hbm_gbs {peak_src}"}
    sv_roof = {"kernel": ("hierarchical-inverse products (hinv_t_kernel + hinv_r_kernel, L^-1 then U^-1)" if hinv
                          else "exec_kernel<1> (H-triangular solve schedule)"),
               "bound": "hbm", "achieved": sv_gbs, "peak": hbm, "unit": "GB/s", "frac": sv_gbs / hbm,
               "traffic": None, "algorithmic_bytes": st["lu_bytes"], "ms": sv_ms, "per_bench_step_ms": n_sv * sv_ms,
               "peak_source": f"hbm_gbs {peak_src}"}
    # the H-LU's GEMM tiles compute in double-float arithmetic on the FP32 pipes:
    # 10 FP32 instructions per FP64-equivalent multiply-add, so the ALU peak is
    # 128 FP32 lanes x SMs x clock / 10 multiply-adds (2 flop each)
    df_peak = df_alu_peak(clocks)
    lu_tf = 2.0 * st["factor_fma"] / (st["factor_ms"] * 1e-3) / 1e12 if st["factor_ms"] > 0 else 0.0
    lu_roof = {"kernel": "exec_kernel<0> (H-LU dataflow executor, double-float GEMM tiles)", "bound": "alu",
               "achieved": lu_tf, "peak": df_peak, "unit": "TFLOP/s", "frac": lu_tf / df_peak, "traffic": None,
               "algorithmic_flops": 2.0 * st["factor_fma"], "ms": st["factor_ms"], "per_bench_step_ms": st["factor_ms"],
               "peak_source": DF_PEAK_SOURCE,
               "note": "latency-bound: the planned critical path (chain of diagonal leaf LUs) is about the measured time"}
    parts = [lu_roof, mv_roof, sv_roof]
    roofline = max(parts, key=lambda r: r["per_bench_step_ms"])

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "mixed_fp32": "f64+f32", "mixed_bf16": "f64+bf16"}[opts["precision"]],
            "data": "synthetic",
            "config": {"workload": name, "N": N, "cn_steps": cn_steps, "dt": dt, "leaf": opts["leaf"],
                       "aca_tol": opts["aca_tol"], "max_rank": opts["max_rank"],
                       "lu_max_rank": opts["lu_max_rank"], "refine_sweeps": opts["refine_max"],
                       "precision": opts["precision"], "solve": opts["solve"], "cn_form": opts["cn_form"],
                       "parallelism": f"replicas x{world}",
                       "l2": f"working set (H + factors, {(st['h_bytes'] + st['lu_bytes']) / 1e9:.1f} GB) "
                             "exceeds L2; no flush needed"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "solve_roofline": sv_roof, "matvec_roofline": mv_roof, "factor_roofline": lu_roof,
            "accuracy": {"rel_l2_vs_dense_fp64_oracle": oracle_err, "oracle_reference": oracle_ref,
                         "rel_l2_vs_converged_fp64_solves": rel_err,
                         "reference": f"same H-matrix CN run at N={N} with 3 FP64 refinement sweeps per step"},
            "stats": {k: st[k] for k in ("h_bytes", "lu_bytes", "max_rank_seen", "lu_max_rank_seen",
                                         "dense_blocks", "lowrank_blocks", "last_refine_resid", "solve_mode",
                                         "hinv_max_rank", "hinv_capped", "hinv_ms", "factor_ms", "factor_fma",
                                         "device_bytes")}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample() if prob["dim"] == 1 else cpu_sample_2d(name)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
