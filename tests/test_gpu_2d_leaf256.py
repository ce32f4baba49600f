"""The 2D fractional Laplacian workload's own path against the dense FP64
oracle: leaf 256 (the leaf-256 near field), ACA tolerance 1e-8 and rank <= 64,
factor rank <= 16, no refinement sweeps, the substitution solve on solve
blocks of <= 1024 rows, identity-form CN steps of dt = 1/200 from the
Gaussian bump (sigma = 0.1), as the 2D bench runs them, at grid sides the
dense oracle reaches (64 and 80) and for both orders of the workload
(s = 0.3 and 0.75).  20 steps, relative L2 <= 1e-8."""
import numpy as np
import pytest

from oracle import levy_dense as O
from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu

pytestmark = pytest.mark.gpu

CASES = [(64, 0.3), (80, 0.75)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("n,s", CASES, ids=[f"n{n}_s{s}" for n, s in CASES])
def test_frac2d_leaf256_against_oracle(n, s):
    prob = W.frac_lap_2d(n, s)
    _, opts, dt, _, kind = W.WORKLOADS["frac_lap_2d_256x256_s0.75"]
    opts = dict(opts, lu_max_rank=16, lu_tol=1e-10, refine_max=0)
    steps = 20
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    st = H.stats(F)
    assert st["solve_mode"] == hmat.HM_SOLVE_SUBST
    assert st["dense_blocks"] > 0 and st["lowrank_blocks"] > 0
    u0 = W.initial_data(prob, kind)
    u = dev(u0)
    hmat.cn_solve(H, F, dt, steps, u)
    ref = O.cn_solve(O.generator_dense(prob), u0, dt, steps)
    err = np.linalg.norm(host(u) - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, err
    F.free()
    H.free()
