"""The 2D fractional Laplacian workload's own path against the dense FP64
oracle: leaf 256 (the leaf-256 near field), ACA tolerance 1e-8 and rank <= 64,
factor rank <= 16, no refinement sweeps, the substitution solve on solve
blocks of <= 1024 rows, identity-form CN steps of dt = 1/200 from the
Gaussian bump (sigma = 0.1), as the 2D bench runs them, at grid sides the
dense oracle reaches (64 and 80) and for both orders of the workload
(s = 0.3 and 0.75).  20 steps, relative L2 <= 1e-8.  At side 128 (N = 16384)
the full 200 steps against the dense oracle solution stored by
``tests/golden/make_frac2d_golden.py``."""
import os

import numpy as np
import pytest

from oracle import levy_dense as O
from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu

pytestmark = pytest.mark.gpu

CASES = [(64, 0.3), (80, 0.75)]
GOLD128 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "frac2d_n128_s0.75_dt5e-3.npz")


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


def test_frac2d_leaf256_side128_full_run_against_stored_oracle():
    """The bench's own options, dt and step count (200 steps of 1/200) at side
    128, where the host's dense LU still fits: u after 20 and 200 steps
    against the stored oracle solution, relative L2 <= 1e-8."""
    g = np.load(GOLD128)
    prob, opts, dt, steps, kind = W.WORKLOADS["frac_lap_2d_256x256_s0.75"]
    prob = W.frac_lap_2d(128, 0.75)
    opts = dict(opts, lu_max_rank=16, lu_tol=1e-10, refine_max=0)
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    assert H.stats(F)["solve_mode"] == hmat.HM_SOLVE_SUBST
    u = dev(W.initial_data(prob, kind))
    hmat.cn_solve(H, F, dt, 20, u)
    err20 = np.linalg.norm(host(u) - g["u20"]) / np.linalg.norm(g["u20"])
    hmat.cn_solve(H, F, dt, steps - 20, u, step0=20)
    err = np.linalg.norm(host(u) - g[f"u{steps}"]) / np.linalg.norm(g[f"u{steps}"])
    F.free()
    H.free()
    assert err20 <= 1e-8 and err <= 1e-8, (err20, err)
