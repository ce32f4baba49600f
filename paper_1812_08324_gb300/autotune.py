"""Leaf-size autotuner for batched solves.

For one representative problem per size bucket (N rounded to a power of two)
it builds the H-matrix, factors I - dt/2 G and times a few CN steps for each
candidate leaf size on the GPU, then keeps the leaf that minimises the
projected run time  factor + steps x (time per CN step).  Results are cached
per (dim, bucket, candidates, steps) for the life of the process.

    from paper_1812_08324_gb300 import autotune
    leafs = autotune.tune_batch(batch, dt, steps)      # one leaf per problem
"""
from __future__ import annotations

import math
import time

from . import hmat

_CACHE: dict = {}


def _sync():
    import torch
    torch.cuda.synchronize()


def tune_leaf(prob: dict, opts: dict, dt: float, steps: int, candidates=(64, 128, 256), probe_steps: int = 5):
    """Best leaf for this problem and the timing table {leaf: (factor_s, step_s)}."""
    import torch
    from . import workloads as W

    table = {}
    u0 = W.gaussian_u0(prob, 50.0) if prob["dim"] == 1 else W.bump_u0(prob)
    for leaf in candidates:
        if leaf > max(prob["n"][0] * (prob["n"][1] if prob["dim"] == 2 else 1), 1):
            continue
        o = dict(opts, leaf=int(leaf))
        _sync()
        t0 = time.perf_counter()
        H = hmat.HMatrix(prob, o)
        F = H.factor(-0.5 * dt)
        _sync()
        t1 = time.perf_counter()
        u = torch.tensor(u0, dtype=torch.float64, device="cuda")
        hmat.cn_solve(H, F, dt, 1, u)          # warm-up
        _sync()
        t2 = time.perf_counter()
        hmat.cn_solve(H, F, dt, probe_steps, u)
        _sync()
        t3 = time.perf_counter()
        table[int(leaf)] = (t1 - t0, (t3 - t2) / probe_steps)
        F.free()
        H.free()
    best = min(table, key=lambda l: table[l][0] + steps * table[l][1])
    return best, table


def _bucket(prob: dict) -> int:
    n = prob["n"][0] * (prob["n"][1] if prob["dim"] == 2 else 1)
    return int(round(math.log2(max(n, 1))))


def tune_batch(batch, dt: float, steps: int, candidates=(64, 128, 256), probe_steps: int = 5):
    """One leaf per (problem, options) of the batch: each size bucket is tuned
    once on its first problem; returns the list of leaf sizes."""
    out = []
    for prob, opts in batch:
        key = (prob["dim"], _bucket(prob), tuple(candidates), int(steps))
        if key not in _CACHE:
            _CACHE[key] = tune_leaf(prob, opts, dt, steps, candidates, probe_steps)[0]
        out.append(_CACHE[key])
    return out
