"""Failure detection and resume on the GPU, in the forms that fault no GPU.

* Bounded waits: every dependency wait of the persistent dataflow executor
  gives up after a time limit, sets an error bit that the host reads, and the
  CTA returns.  The test shortens the limit (HM_WAIT_LIMIT_MS) and makes one
  op of the H-LU schedule require one task more than it has
  (HM_TEST_STALL_OP, a host-side edit of the uploaded schedule), so that its
  consumers' waits can only run out.  hm_factor must then return
  HM_ERR_TIMEOUT within a bounded wall time, and a fresh build on the same
  context must factor and solve normally.
* Resume: a Crank-Nicolson state is (u, level); cn_solve from a saved level
  continues the run bit for bit.
"""
import time

import numpy as np
import pytest

from oracle import levy_dense as O
from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu

pytestmark = pytest.mark.gpu

PROB = W.levy_1d(2047)
OPTS = W.default_opts(leaf=128, aca_tol=1e-10, max_rank=32, lu_tol=1e-10, lu_max_rank=32)
DT = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_stalled_dependency_times_out_and_context_survives(monkeypatch):
    H = hmat.HMatrix(PROB, OPTS)
    H.sync()
    monkeypatch.setenv("HM_PIPELINE", "0")        # one schedule: op 0 is the first copy into the factors
    monkeypatch.setenv("HM_WAIT_LIMIT_MS", "50")
    monkeypatch.setenv("HM_TEST_STALL_OP", "0")
    t0 = time.time()
    with pytest.raises(hmat.HMError) as ei:
        H.factor(-0.5 * DT)
    wall = time.time() - t0
    assert ei.value.status == -6, ei.value  # HM_ERR_TIMEOUT
    # each CTA gives up after at most one expired 50 ms wait and returns
    assert wall < 30.0, wall
    H.free()
    monkeypatch.delenv("HM_TEST_STALL_OP")
    monkeypatch.delenv("HM_WAIT_LIMIT_MS")
    monkeypatch.delenv("HM_PIPELINE")
    # the context is usable: a fresh build factors and solves, and matches the oracle
    H2 = hmat.HMatrix(PROB, OPTS)
    F2 = H2.factor(-0.5 * DT)
    H2.sync()
    G = O.generator_dense(PROB)
    M = np.eye(G.shape[0]) - 0.5 * DT * G
    b = np.random.default_rng(3).standard_normal(G.shape[0])
    x = host(F2.solve(dev(b)))
    ref = np.linalg.solve(M, b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8
    F2.free()
    H2.free()


@pytest.mark.parametrize("refine", [0, 2])
def test_resume_from_saved_level_is_bitwise(refine):
    """cn_solve for 2k steps equals cn_solve for k steps followed by cn_solve
    for k steps from step0 = k (with forcing, whose levels are relative to
    step0), bit for bit; with and without refinement sweeps."""
    H = hmat.HMatrix(PROB, dict(OPTS, refine_max=refine))
    F = H.factor(-0.5 * DT)
    N = H.n
    x = W.coords(PROB)[:, 0]
    u0 = W.gaussian_u0(PROB, 50.0)
    k = 7
    fall = np.stack([np.sin(3 * x) * (1.0 + 0.1 * j) for j in range(2 * k + 1)])
    ua = dev(u0)
    hmat.cn_solve(H, F, DT, 2 * k, ua, dev(fall))
    ub = dev(u0)
    hmat.cn_solve(H, F, DT, k, ub, dev(fall[: k + 1]))
    hmat.cn_solve(H, F, DT, k, ub, dev(fall[k:]), step0=k)
    assert np.array_equal(host(ua), host(ub))
    # no forcing: the graph-replay path (refine 0) resumes bit for bit too
    uc = dev(u0)
    hmat.cn_solve(H, F, DT, 2 * k, uc)
    ud = dev(u0)
    hmat.cn_solve(H, F, DT, k, ud)
    hmat.cn_solve(H, F, DT, k, ud, step0=k)
    assert np.array_equal(host(uc), host(ud))
    assert N == u0.size
    F.free()
    H.free()
