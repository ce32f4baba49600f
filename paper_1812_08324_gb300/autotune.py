"""Autotuner for batched solves: leaf size, triangular-solve mode and
substitution block size.

For one representative problem per size bucket (N rounded to a power of two)
it builds the H-matrix, factors I - dt/2 G and times a few CN steps for each
candidate configuration on the GPU, then keeps the configuration that
minimises the projected run time  factor + steps x (time per CN step).  The
candidates are every leaf size with
  * the hierarchical inverses of the factors (1D problems on a box), and
  * the substitution solve with each candidate solve-block size (rows of the
    largest solve block; block sizes not below N are skipped).
The GEMM tile shapes of the H-LU follow from each operation's output shape
inside the planner and are not searched.  Results are cached per (dim,
bucket, candidates, steps, options) for the life of the process.

    from paper_1812_08324_gb300 import autotune
    cfgs = autotune.tune_batch_configs(batch, dt, steps)  # one options override per problem
    leafs = autotune.tune_batch(batch, dt, steps)         # leaf only (solve mode fixed by opts)
"""
from __future__ import annotations

import math
import time

from . import hmat

_CACHE: dict = {}


def _sync():
    import torch
    torch.cuda.synchronize()


def _n(prob: dict) -> int:
    return prob["n"][0] * (prob["n"][1] if prob["dim"] == 2 else 1)


def _probe(prob: dict, o: dict, dt: float, probe_steps: int):
    """(factor seconds, seconds per CN step) of one configuration."""
    import torch
    from . import workloads as W

    u0 = W.gaussian_u0(prob, 50.0) if prob["dim"] == 1 else W.bump_u0(prob)
    _sync()
    t0 = time.perf_counter()
    H = hmat.HMatrix(prob, o)
    F = H.factor(-0.5 * dt)
    _sync()
    t1 = time.perf_counter()
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    hmat.cn_solve(H, F, dt, 1, u)          # warm-up (records the step's graph)
    _sync()
    t2 = time.perf_counter()
    hmat.cn_solve(H, F, dt, probe_steps, u)
    _sync()
    t3 = time.perf_counter()
    F.free()
    H.free()
    return t1 - t0, (t3 - t2) / probe_steps


def configurations(prob: dict, opts: dict, leafs=(64, 128, 256), solve_blocks=(1024, 2048)):
    """Candidate option overrides for this problem (see the module docstring).
    A `solve` other than "auto" in opts fixes the solve mode."""
    n = _n(prob)
    fixed = opts.get("solve", "auto")
    hinv_ok = prob["dim"] == 1 and prob.get("domain", 0) == 0
    out = []
    for leaf in leafs:
        if leaf > max(n, 1):
            continue
        if fixed in ("auto", "hinv") and (hinv_ok or fixed == "hinv"):
            out.append({"leaf": int(leaf), "solve": "hinv"})
        if fixed in ("auto", "subst"):
            blocks = [b for b in solve_blocks if b < n] or [0]
            for b in blocks:
                out.append({"leaf": int(leaf), "solve": "subst", "solve_block": int(b)})
    if opts.get("precision", "fp64") != "fp64":  # the mixed precisions need the inverses
        out = [c for c in out if c["solve"] == "hinv"]
    if not out:
        raise ValueError("no solve configuration fits this problem with these options "
                         f"(dim {prob['dim']}, precision {opts.get('precision', 'fp64')}, solve {fixed})")
    return out


def tune_config(prob: dict, opts: dict, dt: float, steps: int, leafs=(64, 128, 256), solve_blocks=(1024, 2048),
                probe_steps: int = 5):
    """Best options override for this problem and the timing table
    {key: (factor_s, step_s)} (key: leaf, solve, solve_block)."""
    table = {}
    best, best_t = None, math.inf
    for cfg in configurations(prob, opts, leafs, solve_blocks):
        f_s, s_s = _probe(prob, dict(opts, **cfg), dt, probe_steps)
        key = (cfg["leaf"], cfg["solve"], cfg.get("solve_block", 0))
        table[key] = (f_s, s_s)
        if f_s + steps * s_s < best_t:
            best, best_t = cfg, f_s + steps * s_s
    return best, table


def tune_leaf(prob: dict, opts: dict, dt: float, steps: int, candidates=(64, 128, 256), probe_steps: int = 5):
    """Best leaf for this problem with the solve mode of opts, and the table
    {leaf: (factor_s, step_s)}."""
    table = {}
    for leaf in candidates:
        if leaf > max(_n(prob), 1):
            continue
        table[int(leaf)] = _probe(prob, dict(opts, leaf=int(leaf)), dt, probe_steps)
    best = min(table, key=lambda l: table[l][0] + steps * table[l][1])
    return best, table


def _bucket(prob: dict) -> int:
    return int(round(math.log2(max(_n(prob), 1))))


def _opts_key(opts: dict):
    return tuple(sorted((k, v) for k, v in opts.items() if k != "leaf" and isinstance(v, (int, float, str))))


def tune_batch_configs(batch, dt: float, steps: int, leafs=(64, 128, 256), solve_blocks=(1024, 2048),
                       probe_steps: int = 5):
    """One options override (leaf, solve, solve_block) per (problem, options)
    of the batch: each size bucket is tuned once, on its first problem."""
    out = []
    for prob, opts in batch:
        key = ("cfg", prob["dim"], _bucket(prob), tuple(leafs), tuple(solve_blocks), int(steps), _opts_key(opts))
        if key not in _CACHE:
            _CACHE[key] = tune_config(prob, opts, dt, steps, leafs, solve_blocks, probe_steps)[0]
        out.append(dict(_CACHE[key]))
    return out


def tune_batch(batch, dt: float, steps: int, candidates=(64, 128, 256), probe_steps: int = 5):
    """One leaf per (problem, options) of the batch, the solve mode as the
    options give it: each size bucket is tuned once on its first problem."""
    out = []
    for prob, opts in batch:
        key = ("leaf", prob["dim"], _bucket(prob), tuple(candidates), int(steps), _opts_key(opts))
        if key not in _CACHE:
            _CACHE[key] = tune_leaf(prob, opts, dt, steps, candidates, probe_steps)[0]
        out.append(_CACHE[key])
    return out
