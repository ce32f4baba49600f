"""Continuous batching: requests that arrive while others run are admitted,
share the device, and every result equals the request solved alone."""
import numpy as np
import pytest

from oracle import levy_dense as O
from paper_1812_08324_gb300 import hmat, serve, workloads as W

from gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _stream():
    # the serving stream's generator at sizes that run in seconds
    return W.serve_stream(8, seed=0, rate=50.0, log2_1d=(9.0, 11.0), sides_2d=(16, 24), steps=(20, 60))


def test_served_results_equal_alone_and_overlap():
    reqs = _stream()
    srv = serve.Server(hbm_budget=50e9, tick_steps=7, realtime=True)
    res = srv.run(reqs)
    assert len(res) == len(reqs)
    overlapped = False
    for r, q in zip(res, reqs):
        H = hmat.HMatrix(q["problem"], q["opts"])
        F = H.factor(-0.5 * q["dt"])
        u = dev(q["u0"])
        hmat.cn_solve(H, F, q["dt"], q["steps"], u)
        assert np.array_equal(host(u), r.u), f"request {q['rid']} differs alone and in the mix"
        assert r.finished >= r.admitted >= 0 and r.latency > 0
        F.free()
        H.free()
    # some request was admitted while another one was still running
    for a in res:
        for b in res:
            if a is not b and b.admitted < a.finished and b.admitted > a.admitted:
                overlapped = True
    assert overlapped
    assert srv.batches_built >= 2 and srv.used == pytest.approx(0.0, abs=1.0)
    s = serve.summary(res)
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_smallest_served_requests_match_oracle():
    """The smallest served request of each kind (1D and 2D) against the dense
    FP64 oracle run of the same problem, initial data, dt and steps: relative
    L2 <= 1e-8."""
    reqs = _stream()
    res = serve.Server(hbm_budget=50e9, tick_steps=7, realtime=False).run(reqs)
    for dim in (1, 2):
        cand = [(r.n, i) for i, (r, q) in enumerate(zip(res, reqs)) if q["problem"]["dim"] == dim]
        assert cand, f"the stream has no {dim}D request"
        _, i = min(cand)
        q = reqs[i]
        G = O.generator_dense(q["problem"])
        ref = O.cn_solve(G, q["u0"], q["dt"], q["steps"])
        err = np.linalg.norm(res[i].u - ref) / np.linalg.norm(ref)
        assert err <= 1e-8, (dim, err)


def test_budget_admits_two_not_three():
    """A budget that holds two requests' estimated footprint but not three:
    at most two requests are ever on the device together, and requests still
    overlap (continuous batching, not a queue)."""
    reqs = [q for q in _stream() if q["problem"]["dim"] == 1][:4]
    est = sorted(serve.estimate_bytes(q) for q in reqs)
    budget = est[-1] + est[-2] + 0.5 * est[0]
    srv = serve.Server(hbm_budget=budget, tick_steps=5, realtime=False)
    res = srv.run(reqs)
    events = sorted([(r.admitted, 1) for r in res] + [(r.finished, -1) for r in res], key=lambda e: (e[0], e[1]))
    live = peak = 0
    for _, d in events:
        live += d
        peak = max(peak, live)
    assert peak == 2, peak


def test_budget_admits_one_at_a_time():
    """A budget below two requests' footprint serialises them (and still
    admits a request that alone exceeds the budget, so nothing starves)."""
    reqs = _stream()[:3]
    srv = serve.Server(hbm_budget=1.0, tick_steps=10, realtime=False)
    res = srv.run(reqs)
    spans = sorted((r.admitted, r.finished) for r in res)
    for (a0, f0), (a1, f1) in zip(spans, spans[1:]):
        assert a1 >= f0 - 1e-6
