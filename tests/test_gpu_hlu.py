"""GPU parity of H-LU, the H-triangular solves and Crank-Nicolson steps
against the dense FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import levy_dense as O
from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu

CASES = [
    ("frac1d_n1023", W.frac_lap_1d(1023, 0.5), W.default_opts(leaf=64, aca_tol=1e-10, max_rank=40,
                                                                lu_tol=1e-10, lu_max_rank=40), 1e-3),
    ("levy1d_n2047", W.levy_1d(2047), W.default_opts(leaf=128, aca_tol=1e-10, max_rank=32,
                                                       lu_tol=1e-10, lu_max_rank=32), 1e-3),
    ("frac2d_n24", W.frac_lap_2d(24, 0.75), W.default_opts(leaf=36, aca_tol=1e-9, max_rank=32,
                                                            lu_tol=1e-10, lu_max_rank=32), 5e-3),
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("name,prob,opts,dt", CASES, ids=[c[0] for c in CASES])
def test_hlu_solve_matches_dense(name, prob, opts, dt):
    """(LU)^{-1} b from the H-LU factors equals the dense solve of I - dt/2 G
    to the accuracy of the compression (no refinement involved)."""
    G = O.generator_dense(prob)
    N = G.shape[0]
    M = np.eye(N) - 0.5 * dt * G
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    H.sync()
    rng = np.random.default_rng(11)
    for b in (rng.standard_normal(N), W.gaussian_u0(prob, 30.0)):
        x = host(F.solve(dev(b)))
        ref = np.linalg.solve(M, b)
        err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
        # the compression tolerances are 1e-10: the factors solve to ~1e-11
        assert err < 1e-8, err
    st = H.stats(F)
    assert st["lu_bytes"] > 0


@pytest.mark.parametrize("name,prob,opts,dt", CASES, ids=[c[0] for c in CASES])
def test_cn_step_matches_oracle(name, prob, opts, dt):
    """One CN step with refinement agrees with the dense oracle to 1e-10."""
    G = O.generator_dense(prob)
    N = G.shape[0]
    H = hmat.HMatrix(prob, dict(opts, refine_max=3))
    F = H.factor(-0.5 * dt)
    u0 = W.gaussian_u0(prob, 30.0) if prob["dim"] == 1 else W.bump_u0(prob)
    f0, f1 = np.sin(np.arange(N) * 0.01), np.cos(np.arange(N) * 0.02)
    u1 = host(hmat.cn_step(H, F, dt, dev(u0), dev(f0), dev(f1)))
    ref = O.cn_solve(G, u0, dt, 1, forcing=lambda k: f0 if k == 0 else f1)
    err = np.linalg.norm(u1 - ref) / np.linalg.norm(ref)
    assert err < 1e-10, err


def test_cn_solve_manufactured_frac1d():
    """Workload 1 (N = 1023, s = 1/2, manufactured (1-x^2)^s e^{-t}): 100 steps of
    the H path against 100 steps of the dense oracle: relative L2 <= 1e-8."""
    prob, opts, dt, steps, kind = W.WORKLOADS["frac_lap_1d_n1023"]
    opts = dict(opts, max_rank=40, lu_max_rank=40, refine_max=3)
    u0, ffun, uex = W.manufactured_unit_ball(prob)
    N = u0.size
    G = O.generator_dense(prob)
    ref = O.cn_solve(G, u0, dt, steps, forcing=lambda k: ffun(k * dt))
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    fall = np.stack([ffun(k * dt) for k in range(steps + 1)])
    u = dev(u0)
    hmat.cn_solve(H, F, dt, steps, u, dev(fall))
    got = host(u)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-8, err
    # and the discrete solution tracks the manufactured one
    assert np.linalg.norm(got - uex(steps * dt)) / np.linalg.norm(uex(steps * dt)) < 1e-3


def test_factor_rejects_mismatched_dt():
    prob, opts, dt, steps, kind = W.WORKLOADS["frac_lap_1d_n1023"]
    H = hmat.HMatrix(prob, dict(opts, max_rank=40, lu_max_rank=40))
    F = H.factor(-0.5 * dt)
    u = dev(np.zeros(prob["n"][0]))
    with pytest.raises(hmat.HMError):
        hmat.cn_step(H, F, 2 * dt, u)


@pytest.mark.slow
def test_hlu_solve_accuracy_full_size_levy1d():
    """1D Levy generator at N = 65536 (leaf 256, ACA rank <= 32, factor rank
    <= 16, dt = 1e-3): one H-LU solve of a random right-hand side agrees with
    its iteratively refined solution (FP64 H-matvec residuals) to 1e-9, and the
    refined solution leaves a relative residual below 1e-12 in the H system.
    A property that holds at any size; the dense oracle does not reach N = 65536."""
    prob, opts, dt, steps, kind = W.WORKLOADS["levy_1d_n65536"]
    H = hmat.HMatrix(prob, dict(opts, lu_max_rank=16, lu_tol=1e-10))
    F = H.factor(-0.5 * dt)
    N = prob["n"][0]
    rng = np.random.default_rng(5)
    b = dev(rng.standard_normal(N))

    def apply_m(x):  # (I - dt/2 G) x = 2x - (I + dt/2 G) x
        return 2 * x - H.matvec(x, alpha=1.0, beta=0.5 * dt)

    x0 = F.solve(b)
    x = x0.clone()
    for _ in range(4):
        x = x + F.solve(b - apply_m(x))
    err = (torch.linalg.norm(x0 - x) / torch.linalg.norm(x)).item()
    res = (torch.linalg.norm(b - apply_m(x)) / torch.linalg.norm(b)).item()
    assert err < 1e-9, err
    assert res < 1e-12, res
    F.free()
    H.free()


@pytest.mark.parametrize("name,prob,opts,dt", CASES, ids=[c[0] for c in CASES])
def test_streamed_factor_equals_unstreamed(name, prob, opts, dt, monkeypatch):
    """Planning streamed into execution in small slices (many launches, ops
    whose producers ran in earlier launches) gives the same factors bit for
    bit as one schedule planned in full before it runs."""
    H = hmat.HMatrix(prob, opts)
    b = dev(np.random.default_rng(2).standard_normal(H.n))
    monkeypatch.setenv("HM_PIPELINE", "0")
    F0 = H.factor(-0.5 * dt)
    x0 = host(F0.solve(b))
    F0.free()
    monkeypatch.setenv("HM_PIPELINE", "1")
    monkeypatch.setenv("HM_CHUNK_OPS", "257")
    F1 = H.factor(-0.5 * dt)
    x1 = host(F1.solve(b))
    F1.free()
    monkeypatch.delenv("HM_CHUNK_OPS")
    H.free()
    assert np.array_equal(x0, x1)


@pytest.mark.parametrize("name,prob,opts,dt", CASES, ids=[c[0] for c in CASES])
def test_double_float_gemm_matches_fp64(name, prob, opts, dt, monkeypatch):
    """The H-LU's GEMM tiles in double-float arithmetic (operands split into
    two floats, 2^-47 relative, sums by two-sum; the default) and the leaf
    LUs in double-float (HM_LU_DF=1; FP64 is the default) agree with the same
    operations in FP64 to far below the compression tolerances (substitution
    solves: the inverses' own truncation would blur the comparison)."""
    H = hmat.HMatrix(prob, dict(opts, solve="subst"))
    b = dev(np.random.default_rng(4).standard_normal(H.n))
    monkeypatch.setenv("HM_GEMM_FP64", "1")
    monkeypatch.setenv("HM_LU_DF", "0")
    F0 = H.factor(-0.5 * dt)
    x0 = host(F0.solve(b))
    F0.free()
    monkeypatch.setenv("HM_GEMM_FP64", "0")
    monkeypatch.setenv("HM_LU_DF", "1")
    F1 = H.factor(-0.5 * dt)
    x1 = host(F1.solve(b))
    F1.free()
    H.free()
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) < 1e-12
