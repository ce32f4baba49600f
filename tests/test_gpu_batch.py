"""Batched factorisation and CN steps: every problem's result equals the
one-problem path bit for bit, and a small member matches the dense oracle."""
import numpy as np
import pytest

from oracle import levy_dense as O
from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _small_batch(count=6):
    # the batched workload's parameter stream at sizes the oracle can check
    return W.levy_batch(count, seed=0, log2_lo=8.0, log2_hi=11.0)


def test_factor_batch_equals_single():
    batch = _small_batch()
    dt = W.LEVY_BATCH_DT
    Hs = [hmat.HMatrix(p, o) for p, o in batch]
    Fb = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
    rng = np.random.default_rng(3)
    for H, Fi in zip(Hs, Fb):
        F1 = H.factor(-0.5 * dt)
        b = dev(rng.standard_normal(H.n))
        x1 = host(F1.solve(b))
        xb = host(Fi.solve(b))
        assert np.array_equal(x1, xb)
        assert H.stats(Fi)["lu_max_rank_seen"] == H.stats(F1)["lu_max_rank_seen"]


def test_inverses_do_not_depend_on_the_construction_grouping(monkeypatch):
    """A batch's hierarchical inverses are built with the construction steps
    of several problems merged into shared launches (groups of stacked rows);
    the solves they give are the same bit for bit whether every problem is
    alone in its group, a few share one, or all share one."""
    batch = _small_batch(8)
    dt = W.LEVY_BATCH_DT
    Hs = [hmat.HMatrix(p, o) for p, o in batch]
    rng = np.random.default_rng(5)
    bs = [dev(rng.standard_normal(H.n)) for H in Hs]
    sols = []
    for rows in (None, "1", "2500"):
        if rows is None:
            monkeypatch.delenv("HM_HINV_GROUP_ROWS", raising=False)
        else:
            monkeypatch.setenv("HM_HINV_GROUP_ROWS", rows)
        Fs = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
        assert all(H.stats(F)["solve_mode"] == hmat.HM_SOLVE_HINV for H, F in zip(Hs, Fs))
        sols.append([host(F.solve(b)) for F, b in zip(Fs, bs)])
        for F in Fs:
            F.free()
    for other in sols[1:]:
        for x0, x1 in zip(sols[0], other):
            assert np.array_equal(x0, x1)


def test_factor_batch_in_many_small_launches_is_identical(monkeypatch):
    """The streamed H-LU with small planner chunks and a small cap on the ops
    of one launch (each problem's chunks spread over many launches, taken
    round robin over the problems) gives the same solves bit for bit as the
    default slicing."""
    batch = _small_batch(6)
    dt = W.LEVY_BATCH_DT
    Hs = [hmat.HMatrix(p, o) for p, o in batch]
    rng = np.random.default_rng(9)
    bs = [dev(rng.standard_normal(H.n)) for H in Hs]
    sols = []
    for chunk, cap in ((None, None), ("700", "2000")):
        for k, v in (("HM_CHUNK_OPS", chunk), ("HM_SLICE_OPS", cap)):
            if v is None:
                monkeypatch.delenv(k, raising=False)
            else:
                monkeypatch.setenv(k, v)
        Fs = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
        sols.append([host(F.solve(b)) for F, b in zip(Fs, bs)])
        for F in Fs:
            F.free()
    for x0, x1 in zip(*sols):
        assert np.array_equal(x0, x1)


def test_factor_with_64x64_gemm_tiles_is_identical(monkeypatch):
    """GEMMs run as 64 x 64 output tiles (HM_GEMM_BIG_TILES=1 and
    HM_GEMM_BIG_WAVE=0: every GEMM that is not narrow, in every wave) give the
    same factors bit for bit as 32 x 32 tiles: every output sums its k terms
    in the same order whatever the tile; 1D members and a 2D problem."""
    batch = _small_batch(4) + [(W.frac_lap_2d(40, 0.6), W.default_opts(leaf=64, aca_tol=1e-8, max_rank=32,
                                                                         lu_max_rank=16, refine_max=0))]
    dt = W.LEVY_BATCH_DT
    Hs = [hmat.HMatrix(p, o) for p, o in batch]
    rng = np.random.default_rng(11)
    bs = [dev(rng.standard_normal(H.n)) for H in Hs]
    sols = []
    for big in ("0", "1"):
        monkeypatch.setenv("HM_GEMM_BIG_TILES", big)
        monkeypatch.setenv("HM_GEMM_BIG_WAVE", "0")
        Fs = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
        sols.append([host(F.solve(b)) for F, b in zip(Fs, bs)])
        for F in Fs:
            F.free()
    for x0, x1 in zip(*sols):
        assert np.array_equal(x0, x1)


def test_cn_solve_batch_equals_single_and_oracle():
    batch = _small_batch()
    dt, steps = W.LEVY_BATCH_DT, 20
    Hs = [hmat.HMatrix(p, o) for p, o in batch]
    Fs = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
    u0s = [W.gaussian_u0(p, 50.0) for p, _ in batch]
    ub = [dev(u) for u in u0s]
    hmat.cn_solve_batch(Hs, Fs, dt, steps, ub)
    torch.cuda.synchronize()
    for H, F, u0, u in zip(Hs, Fs, u0s, ub):
        us = dev(u0)
        hmat.cn_solve(H, F, dt, steps, us)
        assert np.array_equal(host(us), host(u)), "batched CN differs from the single path"
    # the smallest member against the dense oracle
    i = int(np.argmin([p["n"][0] for p, _ in batch]))
    G = O.generator_dense(batch[i][0])
    ref = O.cn_solve(G, u0s[i], dt, steps)
    err = np.linalg.norm(host(ub[i]) - ref) / np.linalg.norm(ref)
    assert err < 1e-8, err


def test_cn_solve_batch_mixed_1d_2d_with_refinement():
    """A 2D member exercises the Morton gather/scatter; one refinement sweep
    exercises the residual path; results still equal the single path."""
    dt, steps = 1e-3, 5
    probs = [(W.frac_lap_2d(24, 0.75), W.default_opts(leaf=36, aca_tol=1e-9, max_rank=32, lu_max_rank=32,
                                                        refine_max=1)),
             (W.levy_1d(700, sigma=0.3, b=-0.4, alpha=1.2), W.default_opts(leaf=64, max_rank=32, lu_max_rank=16,
                                                                             refine_max=1))]
    Hs = [hmat.HMatrix(p, o) for p, o in probs]
    Fs = [H.factor(-0.5 * dt) for H in Hs]
    u0s = [W.bump_u0(probs[0][0]), W.gaussian_u0(probs[1][0], 50.0)]
    ub = [dev(u) for u in u0s]
    hmat.cn_solve_batch(Hs, Fs, dt, steps, ub)
    torch.cuda.synchronize()
    for H, F, u0, u in zip(Hs, Fs, u0s, ub):
        us = dev(u0)
        hmat.cn_solve(H, F, dt, steps, us)
        assert np.array_equal(host(us), host(u))


def test_cn_solve_batch_rejects_bad_input():
    batch = _small_batch(2)
    dt = W.LEVY_BATCH_DT
    Hs = [hmat.HMatrix(p, o) for p, o in batch]
    Fs = hmat.factor_batch(Hs, [-0.5 * dt] * 2)
    us = [dev(W.gaussian_u0(p, 50.0)) for p, _ in batch]
    with pytest.raises(hmat.HMError):      # factors of another dt
        hmat.cn_solve_batch(Hs, Fs, 2 * dt, 3, us)
    with pytest.raises(hmat.HMError):      # the same problem twice
        hmat.cn_solve_batch([Hs[0], Hs[0]], [Fs[0], Fs[0]], dt, 3, us)


def test_autotune_configs_cover_leaf_solve_and_block():
    """The autotuner's search space for a 1D problem holds the inverses and the
    substitution solve with each block size below N, and its choice is one of
    them; the batch with the chosen options matches the oracle."""
    from paper_1812_08324_gb300 import autotune
    batch = _small_batch(2)
    dt = W.LEVY_BATCH_DT
    p0, o0 = batch[0]
    cands = autotune.configurations(p0, o0, leafs=(32, 64), solve_blocks=(256, 512))
    kinds = {(c["solve"], c.get("solve_block", 0)) for c in cands}
    assert ("hinv", 0) in kinds and ("subst", 256) in kinds
    cfgs = autotune.tune_batch_configs(batch, dt, 50, leafs=(32, 64), solve_blocks=(256, 512), probe_steps=2)
    tuned = [(p, dict(o, **c)) for (p, o), c in zip(batch, cfgs)]
    for c, (p, o) in zip(cfgs, batch):
        assert c in autotune.configurations(p, o, leafs=(32, 64), solve_blocks=(256, 512))
    Hs = [hmat.HMatrix(p, o) for p, o in tuned]
    Fs = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
    us = [dev(W.gaussian_u0(p, 50.0)) for p, _ in tuned]
    hmat.cn_solve_batch(Hs, Fs, dt, 10, us)
    for (p, o), u in zip(tuned, us):
        ref = O.cn_solve(O.generator_dense(p), W.gaussian_u0(p, 50.0), dt, 10)
        assert np.linalg.norm(host(u) - ref) / np.linalg.norm(ref) < 1e-8


def test_autotune_picks_a_candidate_and_batch_stays_exact():
    from paper_1812_08324_gb300 import autotune
    batch = _small_batch(3)
    dt = W.LEVY_BATCH_DT
    leafs = autotune.tune_batch(batch, dt, 50, candidates=(32, 64), probe_steps=2)
    assert all(l in (32, 64) for l in leafs)
    tuned = [(p, dict(o, leaf=l)) for (p, o), l in zip(batch, leafs)]
    Hs = [hmat.HMatrix(p, o) for p, o in tuned]
    Fs = hmat.factor_batch(Hs, [-0.5 * dt] * len(Hs))
    us = [dev(W.gaussian_u0(p, 50.0)) for p, _ in tuned]
    hmat.cn_solve_batch(Hs, Fs, dt, 10, us)
    assert hmat.batch_graphed()
    for (p, o), u in zip(tuned, us):
        G = O.generator_dense(p)
        ref = O.cn_solve(G, W.gaussian_u0(p, 50.0), dt, 10)
        assert np.linalg.norm(host(u) - ref) / np.linalg.norm(ref) < 1e-8
