"""Continuous-batching server for Crank-Nicolson requests.

Requests (problem, options, dt, steps, u0) arrive over time.  The loop admits
waiting requests in arrival order while their device memory fits the HBM
budget (the estimate per unknown, or the measured footprint once larger), builds their H-matrices and factors all newly admitted ones in one
batched H-LU launch (hm_factor_batch), and advances every admitted request
together: each tick runs k CN steps of all active requests through one batch
(one merged solve launch and one batched H-matvec per step, replayed as a CUDA
graph; hm_batch_create / hm_batch_step), with k the smallest remaining step
count capped at tick_steps.  A request that finishes releases its memory at
once, and requests that arrived meanwhile join at the next tick, so their work
overlaps on the device with the requests already running.  Each result equals
the request solved alone bit for bit (the batched kernels do the same
arithmetic in the same order).

    from paper_1812_08324_gb300 import serve, workloads as W
    results = serve.Server(hbm_budget=150e9).run(W.serve_stream(200))
    print(serve.summary(results))
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import hmat

# Device bytes per unknown assumed at admission (H-matrix + what the solves
# read: the factors in 2D, the factors' hierarchical inverses in 1D); a request
# is charged the larger of this and its measured footprint.
EST_BYTES_PER_UNKNOWN = {1: 30e3, 2: 450e3}


@dataclass
class Result:
    rid: int
    n: int
    steps: int
    arrival: float
    admitted: float = 0.0
    finished: float = 0.0
    u: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Slot:
    req: dict
    res: Result
    H: object
    F: object
    u: object
    remaining: int
    bytes: float


def estimate_bytes(req: dict) -> float:
    p = req["problem"]
    n = p["n"][0] * (p["n"][1] if p["dim"] == 2 else 1)
    return EST_BYTES_PER_UNKNOWN[p["dim"]] * n


class Server:
    def __init__(self, hbm_budget: float = 150e9, tick_steps: int = 20, realtime: bool = True):
        self.budget = float(hbm_budget)
        self.tick = int(tick_steps)
        self.realtime = realtime
        self.used = 0.0
        self.peak_used = 0.0
        self.batches_built = 0
        self.ticks = 0

    def run(self, requests) -> list[Result]:
        """Serve the requests (dicts with arrival, problem, opts, dt, steps, u0),
        returning one Result per request in request order.  With realtime the
        arrival times are honoured on the wall clock; otherwise every request
        is visible from the start."""
        import torch

        reqs = sorted(requests, key=lambda r: r["arrival"])
        results = {}
        pending = collections.deque()
        active: list[_Slot] = []
        batch = None
        dirty = False
        i = 0
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while i < len(reqs) or pending or active:
            t = now()
            while i < len(reqs) and (not self.realtime or reqs[i]["arrival"] <= t):
                pending.append(reqs[i])
                i += 1
            # admission in arrival order while the memory estimate fits
            new = []
            while pending and (self.used + estimate_bytes(pending[0]) <= self.budget or not (active or new)):
                r = pending.popleft()
                self.used += estimate_bytes(r)
                new.append(r)
            if new:
                t_adm = now()
                Hs = [hmat.HMatrix(r["problem"], r["opts"]) for r in new]
                Fs = hmat.factor_batch(Hs, [-0.5 * r["dt"] for r in new])
                for r, H, F in zip(new, Hs, Fs):
                    # a request holds the larger of its estimate and its measured
                    # footprint until it finishes
                    charged = max(float(H.stats(F)["device_bytes"]), estimate_bytes(r))
                    self.used += charged - estimate_bytes(r)
                    res = Result(r["rid"], H.n, r["steps"], r["arrival"], admitted=t_adm)
                    u = torch.tensor(r["u0"], dtype=torch.float64, device="cuda")
                    active.append(_Slot(r, res, H, F, u, r["steps"], charged))
                self.peak_used = max(self.peak_used, self.used)
                dirty = True
            if not active:
                if i < len(reqs) and self.realtime:
                    time.sleep(max(0.0, min(0.05, reqs[i]["arrival"] - now())))
                continue
            if dirty:
                if batch is not None:
                    batch.free()
                batch = hmat.Batch([s.H for s in active], [s.F for s in active], [s.req["dt"] for s in active])
                self.batches_built += 1
                dirty = False
            k = min(self.tick, min(s.remaining for s in active))
            batch.step([s.u for s in active], k)
            torch.cuda.synchronize()
            self.ticks += 1
            for s in active:
                s.remaining -= k
            done = [s for s in active if s.remaining == 0]
            if done:
                t_done = now()
                batch.free()
                batch = None
                for s in done:
                    s.res.finished = t_done
                    s.res.u = s.u.cpu().numpy()
                    results[s.res.rid] = s.res
                    s.F.free()
                    s.H.free()
                    self.used -= s.bytes
                active = [s for s in active if s.remaining > 0]
                dirty = True
        if batch is not None:
            batch.free()
        return [results[r["rid"]] for r in requests]


def summary(results: list[Result]) -> dict:
    lat = np.array([r.latency for r in results])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    work = float(sum(r.n * r.steps for r in results))
    return {"requests": len(results), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "span_s": span,
            "unknown_steps_per_s": work / span if span > 0 else float("nan")}
