"""The triangular solves through hierarchical inverses of the H-LU factors
(HM_SOLVE_HINV, the default for 1D problems), their mixed-precision storage
with FP64 refinement, and the substitution solve's large solve blocks, all
against the dense FP64 oracle -- including the 1D Levy workload's own path at
N = 32768 (2048-row solve blocks, leaf 256) against stored oracle solutions
written by ``tests/golden/make_levy1d_golden.py``."""
import os

import numpy as np
import pytest

from oracle import levy_dense as O
from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD32K = os.path.join(HERE, "golden", "levy1d_n32768_dt1e-3.npz")

SMALL = [
    ("frac1d_n1023", W.frac_lap_1d(1023, 0.5), W.default_opts(leaf=64, aca_tol=1e-10, max_rank=40,
                                                                lu_tol=1e-10, lu_max_rank=40), 1e-3),
    ("levy1d_n2047", W.levy_1d(2047), W.default_opts(leaf=128, aca_tol=1e-10, max_rank=32,
                                                       lu_tol=1e-10, lu_max_rank=16), 1e-3),
    ("levy1d_n3001_odd", W.levy_1d(3001, sigma=0.3, b=-0.6, alpha=1.1),
     W.default_opts(leaf=100, aca_tol=1e-10, max_rank=32, lu_tol=1e-10, lu_max_rank=16), 2e-3),
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("name,prob,opts,dt", SMALL, ids=[c[0] for c in SMALL])
def test_hinv_solve_matches_dense(name, prob, opts, dt):
    """(LU)^{-1} b through the inverses equals the dense solve of I - dt/2 G
    to 1e-9 and the substitution solve of the same factors to 1e-10; the
    inverses' ranks stay below the cap and the solve reads fewer bytes than
    the factors."""
    G = O.generator_dense(prob)
    N = G.shape[0]
    M = np.eye(N) - 0.5 * dt * G
    H = hmat.HMatrix(prob, dict(opts, solve="hinv"))
    F = H.factor(-0.5 * dt)
    Hs = hmat.HMatrix(prob, dict(opts, solve="subst"))
    Fs = Hs.factor(-0.5 * dt)
    st = H.stats(F)
    assert st["solve_mode"] == hmat.HM_SOLVE_HINV
    assert 0 < st["hinv_max_rank"] < 40 and st["hinv_capped"] == 0
    assert Hs.stats(Fs)["solve_mode"] == hmat.HM_SOLVE_SUBST
    rng = np.random.default_rng(7)
    for b in (rng.standard_normal(N), W.gaussian_u0(prob, 30.0)):
        x = host(F.solve(dev(b)))
        xs = host(Fs.solve(dev(b)))
        ref = np.linalg.solve(M, b)
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10
    # repeated solves are bitwise reproducible (fixed summation orders)
    b = dev(rng.standard_normal(N))
    assert np.array_equal(host(F.solve(b)), host(F.solve(b)))


@pytest.mark.parametrize("prec,sweeps,tol", [("mixed_fp32", 1, 1e-7), ("mixed_fp32", 2, 1e-9),
                                             ("mixed_bf16", 4, 1e-7)])
def test_mixed_precision_cn_matches_oracle(prec, sweeps, tol):
    """FP32 / BF16 storage of the inverses with FP32 accumulation, won back by
    FP64 refinement sweeps against the FP64 H-matvec residual: 50 CN steps of
    the 1D Levy physics agree with the dense FP64 oracle (1e-6 is the mixed
    criterion; FP32 with one sweep stays well inside it)."""
    prob = W.levy_1d(2047)
    dt, steps = 1e-3, 50
    opts = W.default_opts(leaf=128, aca_tol=1e-10, max_rank=32, lu_tol=1e-10, lu_max_rank=16, precision=prec,
                          refine_max=sweeps)
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    u0 = W.gaussian_u0(prob, 50.0)
    u = dev(u0)
    hmat.cn_solve(H, F, dt, steps, u)
    ref = O.cn_solve(O.generator_dense(prob), u0, dt, steps)
    err = np.linalg.norm(host(u) - ref) / np.linalg.norm(ref)
    assert err < tol, err
    # unrefined, the low-precision inverses alone are visibly less accurate
    H0 = hmat.HMatrix(prob, dict(opts, refine_max=0))
    F0 = H0.factor(-0.5 * dt)
    u = dev(u0)
    hmat.cn_solve(H0, F0, dt, steps, u)
    err0 = np.linalg.norm(host(u) - ref) / np.linalg.norm(ref)
    assert err0 > 10 * err


def test_substitution_with_2048_row_blocks_matches_oracle_small():
    """The substitution solve with 2048-row solve blocks (the layout the
    default rule picks from 32768 unknowns) forced at N = 4095: a solve and 20
    CN steps against the dense oracle."""
    prob = W.levy_1d(4095)
    dt = 1e-3
    opts = W.default_opts(leaf=128, aca_tol=1e-10, max_rank=32, lu_tol=1e-10, lu_max_rank=16, refine_max=0,
                          solve="subst", solve_block=2048)
    G = O.generator_dense(prob)
    N = G.shape[0]
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    b = np.random.default_rng(1).standard_normal(N)
    ref = np.linalg.solve(np.eye(N) - 0.5 * dt * G, b)
    x = host(F.solve(dev(b)))
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9
    u0 = W.gaussian_u0(prob, 50.0)
    u = dev(u0)
    hmat.cn_solve(H, F, dt, 20, u)
    ref = O.cn_solve(G, u0, dt, 20)
    assert np.linalg.norm(host(u) - ref) / np.linalg.norm(ref) < 1e-8


def _levy32k(solve):
    prob = W.levy_1d(32768)
    opts = W.default_opts(leaf=256, aca_tol=1e-10, max_rank=32, lu_tol=1e-10, lu_max_rank=16, refine_max=0,
                          solve=solve)
    return prob, opts


@pytest.mark.parametrize("solve", ["hinv", "subst"])
def test_levy1d_n32768_against_oracle(solve):
    """The 1D Levy workload's physics at N = 32768, leaf 256, ACA rank <= 32,
    factor rank <= 16, no refinement: u after 20 and after 1000 CN steps
    (dt = 1e-3) against the dense oracle's (one 8.6 GB LU, stored by the
    golden script), relative L2 <= 1e-8.  The substitution solve runs here on
    2048-row solve blocks, the layout of the full-size workload."""
    g = np.load(GOLD32K)
    prob, opts = _levy32k(solve)
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5e-3)
    u = dev(W.gaussian_u0(prob, 50.0))
    hmat.cn_solve(H, F, 1e-3, 20, u)
    e20 = np.linalg.norm(host(u) - g["u20"]) / np.linalg.norm(g["u20"])
    hmat.cn_solve(H, F, 1e-3, 980, u, step0=20)
    e1000 = np.linalg.norm(host(u) - g["u1000"]) / np.linalg.norm(g["u1000"])
    assert e20 < 1e-8, e20
    assert e1000 < 1e-8, e1000
    F.free()
    H.free()


def test_batch_of_hinv_problems_equals_single():
    """A batch mixing hierarchical-inverse (1D) and substitution (2D) solves:
    every result equals the single path bit for bit."""
    dt, steps = 1e-3, 6
    probs = [(W.levy_1d(900, sigma=0.3, b=0.5, alpha=1.4), W.default_opts(leaf=64, max_rank=32, lu_max_rank=16,
                                                                           refine_max=0)),
             (W.levy_1d(1500), W.default_opts(leaf=128, max_rank=32, lu_max_rank=16, refine_max=0,
                                              precision="mixed_fp32")),
             (W.frac_lap_2d(20, 0.6), W.default_opts(leaf=36, aca_tol=1e-9, max_rank=32, lu_max_rank=32,
                                                     refine_max=0))]
    # a batch shares refine_max; the FP32 member's accuracy is not the point here
    Hs = [hmat.HMatrix(p, o) for p, o in probs]
    Fs = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
    u0s = [W.gaussian_u0(probs[0][0], 50.0), W.gaussian_u0(probs[1][0], 50.0), W.bump_u0(probs[2][0])]
    ub = [dev(u) for u in u0s]
    hmat.cn_solve_batch(Hs, Fs, dt, steps, ub)
    for H, F, u0, u in zip(Hs, Fs, u0s, ub):
        us = dev(u0)
        hmat.cn_solve(H, F, dt, steps, us)
        assert np.array_equal(host(us), host(u))
    assert [H.stats(F)["solve_mode"] for H, F in zip(Hs, Fs)] == [2, 2, 1]


def test_double_float_construction_matches_fp64(monkeypatch):
    """The inverses' construction products in double-float arithmetic (the
    default) and in FP64 (HM_HINV_BUILD_FP64=1) give the same solves to far
    below the inverses' truncation tolerance, with the same ranks; FP64-storage
    products (HM_HINV_FP64=1) and the float-pair storage agree likewise."""
    prob, opts, dt = SMALL[1][1], dict(SMALL[1][2], solve="hinv"), SMALL[1][3]
    H = hmat.HMatrix(prob, opts)
    b = dev(np.random.default_rng(9).standard_normal(H.n))
    F0 = H.factor(-0.5 * dt)
    x0, r0 = host(F0.solve(b)), H.stats(F0)["hinv_max_rank"]
    F0.free()
    monkeypatch.setenv("HM_HINV_BUILD_FP64", "1")
    F1 = H.factor(-0.5 * dt)
    x1, r1 = host(F1.solve(b)), H.stats(F1)["hinv_max_rank"]
    F1.free()
    monkeypatch.delenv("HM_HINV_BUILD_FP64")
    monkeypatch.setenv("HM_HINV_FP64", "1")
    F2 = H.factor(-0.5 * dt)
    x2 = host(F2.solve(b))
    F2.free()
    H.free()
    assert abs(r0 - r1) <= 1
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) < 1e-11
    assert np.linalg.norm(x2 - x0) / np.linalg.norm(x0) < 1e-12


@pytest.mark.parametrize("form", ["identity", "literal"])
@pytest.mark.parametrize("sweeps", [0, 1])
def test_cn_forms_with_forcing_match_oracle(form, sweeps):
    """Both arrangements of the CN step (cn_form: the identity v = u^n +
    u^{n+1} with no H-matvec, or the right-hand side by the H-matvec as Eq.
    scheme writes it), with and without a refinement sweep, with a time-varying
    forcing: 40 steps against the dense oracle's literal form, relative L2
    <= 1e-9; the two forms agree with each other to 1e-10."""
    prob = W.levy_1d(2047)
    dt, steps = 1e-3, 40
    opts = W.default_opts(leaf=128, aca_tol=1e-10, max_rank=32, lu_tol=1e-10, lu_max_rank=16,
                          refine_max=sweeps, cn_form=form)
    H = hmat.HMatrix(prob, opts)
    F = H.factor(-0.5 * dt)
    N = H.n
    x = np.linspace(-1.0, 1.0, N)
    fs = np.stack([np.cos(3.0 * x + 0.05 * n) * (1.0 + 0.01 * n) for n in range(steps + 1)])
    u0 = W.gaussian_u0(prob, 50.0)
    u = dev(u0)
    hmat.cn_solve(H, F, dt, steps, u, f=dev(fs))
    ref = O.cn_solve(O.generator_dense(prob), u0, dt, steps, forcing=lambda n: fs[n])
    err = np.linalg.norm(host(u) - ref) / np.linalg.norm(ref)
    assert err < 1e-9, err
    # and without forcing (the graph-replay path when sweeps = 0)
    u = dev(u0)
    hmat.cn_solve(H, F, dt, steps, u)
    ref0 = O.cn_solve(O.generator_dense(prob), u0, dt, steps)
    assert np.linalg.norm(host(u) - ref0) / np.linalg.norm(ref0) < 1e-9
    other = "literal" if form == "identity" else "identity"
    H2 = hmat.HMatrix(prob, dict(opts, cn_form=other))
    F2 = H2.factor(-0.5 * dt)
    u2 = dev(u0)
    hmat.cn_solve(H2, F2, dt, steps, u2)
    assert np.linalg.norm(host(u2) - host(u)) / np.linalg.norm(host(u)) < 1e-10
