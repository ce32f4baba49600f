"""Host-side planner (no GPU): the C library loads on a CPU-only machine, exports
every symbol the header declares, and its cluster/block trees satisfy the
definitions of App. "Construction and Storage" checked by brute force."""
import math
import os
import re

import numpy as np
import pytest

from paper_1812_08324_gb300 import build, hmat, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return hmat.load()


def test_exports_every_declared_symbol(lib):
    header = open(os.path.join(ROOT, "include", "levy_hmat.h")).read()
    declared = set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(\w+)\(", header, re.M))
    declared = {d for d in declared if d.startswith(("hm_", "cn_"))}
    assert declared == set(hmat.EXPORTED), declared ^ set(hmat.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def _boxes(perm, dim, n0, row0, m):
    if dim == 1:
        idx = perm[row0:row0 + m][:, None]
    else:
        p = perm[row0:row0 + m]
        idx = np.stack([p % n0, p // n0], axis=1)
    return idx.min(0), idx.max(0) + 1


def _adm(box_a, box_b, eta):
    (la, ha), (lb, hb) = box_a, box_b
    da = float(np.sum((ha - la) ** 2))
    db = float(np.sum((hb - lb) ** 2))
    gap = np.maximum(0, np.maximum(lb - ha, la - hb))
    dist = float(np.sum(gap ** 2))
    return math.sqrt(min(da, db)) <= eta * math.sqrt(dist)


CASES = [
    (W.frac_lap_1d(1023), dict(leaf=64, eta=1.0), (16, 46, 66)),
    (W.levy_1d(4096), dict(leaf=256, eta=1.0), (16, 46, 66)),
    (W.frac_lap_2d(32), dict(leaf=16, eta=1.0), None),
    (W.frac_lap_2d(20), dict(leaf=16, eta=1.0), None),   # non power-of-two side
    (dict(W.frac_lap_2d(24), n=[24, 24]), dict(leaf=10, eta=1.5), None),
]


@pytest.mark.parametrize("prob,opts,expect", CASES)
def test_block_tree_partitions_and_admissibility(prob, opts, expect):
    o = W.default_opts(**opts)
    info = hmat.plan_info(prob, o)
    row0, m, col0, nc, typ, perm = hmat.plan_blocks(prob, o)
    N = info["n"]
    assert sorted(perm.tolist()) == list(range(N))
    # every (row, col) pair lies in exactly one leaf block
    cover = np.zeros((N, N), dtype=np.int32)
    for b in range(len(row0)):
        cover[row0[b]:row0[b] + m[b], col0[b]:col0[b] + nc[b]] += 1
    assert np.all(cover == 1)
    dim, n0 = prob["dim"], prob["n"][0]
    for b in range(len(row0)):
        bt = _boxes(perm, dim, n0, row0[b], m[b])
        bs = _boxes(perm, dim, n0, col0[b], nc[b])
        if typ[b] == 1:
            assert _adm(bt, bs, o["eta"]), b
        else:
            assert typ[b] == 2 and not _adm(bt, bs, o["eta"]) or row0[b] == col0[b]
            assert m[b] <= o["leaf"] and nc[b] <= o["leaf"]
    if expect is not None:
        assert (info["leaves"], info["dense_blocks"], info["lowrank_blocks"]) == expect


def test_paper_scale_block_counts():
    """Counts of the spec configurations (1D: block-tridiagonal near
    field; 2D: 5 x 5 neighbourhood minus its corners per leaf)."""
    i1 = hmat.plan_info(W.levy_1d(65536), W.default_opts(leaf=256))
    assert (i1["leaves"], i1["dense_blocks"], i1["lowrank_blocks"]) == (256, 766, 1482)
    i2 = hmat.plan_info(W.frac_lap_2d(256), W.default_opts(leaf=256))
    assert (i2["leaves"], i2["dense_blocks"], i2["lowrank_blocks"]) == (256, 4692, 13444)


def test_morton_order_2d_is_z_curve():
    row0, m, col0, nc, typ, perm = hmat.plan_blocks(W.frac_lap_2d(4), W.default_opts(leaf=1))
    # Z-order of a 4 x 4 grid (axis 0 fastest in natural numbering)
    z = [0, 1, 4, 5, 2, 3, 6, 7, 8, 9, 12, 13, 10, 11, 14, 15]
    assert perm.tolist() == z


@pytest.mark.parametrize("n,leaf", [(31, 64), (48, 100), (64, 256)])
def test_lshape_block_tree(n, leaf):
    """L-shaped domain: the unknowns are the square's grid points outside the
    closed upper-right quadrant (n^2 - ceil(n/2)^2 of them), the cluster order
    is their Z-curve order, and the leaf blocks tile the matrix with every
    admissible block satisfying the eta condition on the true point boxes."""
    prob = W.lshape_poisson(n)
    o = W.default_opts(leaf=leaf)
    info = hmat.plan_info(prob, o)
    k = (n + 1) // 2
    assert info["n"] == n * n - k * k
    N = info["n"]
    row0, m, col0, nc, typ, perm = hmat.plan_blocks(prob, o)
    assert sorted(perm.tolist()) == list(range(N))
    nat = np.array([i0 + n * i1 for i1 in range(n) for i0 in range(n)
                    if not (2 * (i0 + 1) >= n + 1 and 2 * (i1 + 1) >= n + 1)])
    ij = np.stack([nat % n, nat // n], axis=1)[perm]

    def spread(v):
        out = 0
        for b in range(16):
            out |= ((int(v) >> b) & 1) << (2 * b)
        return out
    codes = [spread(a) | (spread(b) << 1) for a, b in ij]
    assert codes == sorted(codes)
    cover = np.zeros((N, N), dtype=np.int32)
    for b in range(len(row0)):
        cover[row0[b]:row0[b] + m[b], col0[b]:col0[b] + nc[b]] += 1
    assert np.all(cover == 1)
    for b in range(len(row0)):
        rt, cs = ij[row0[b]:row0[b] + m[b]], ij[col0[b]:col0[b] + nc[b]]
        bt = (rt.min(0), rt.max(0) + 1)
        bs = (cs.min(0), cs.max(0) + 1)
        if typ[b] == 1:
            assert _adm(bt, bs, o["eta"]), b


def test_variable_order_arguments_are_checked():
    p = W.lshape_poisson(31)
    with pytest.raises(hmat.HMError):
        hmat.plan_info(dict(p, dim=1, n=[31, 1]), W.default_opts())     # L-shape is 2D
    with pytest.raises(hmat.HMError):
        hmat.plan_info(dict(p, kernel="gauss", eps=1.0), W.default_opts())
    with pytest.raises(hmat.HMError):
        hmat.plan_info(dict(p, c=1.0), W.default_opts())
    with pytest.raises(hmat.HMError):
        hmat.plan_info(dict(p, trunc=1.0), W.default_opts())
    with pytest.raises(hmat.HMError):
        hmat.plan_info(dict(p, domain=7), W.default_opts())
    # constant order on the L-shape is a valid problem
    assert hmat.plan_info(dict(p, s_slope=0.0), W.default_opts())["n"] == 31 * 31 - 16 * 16


def test_bad_arguments_are_rejected(lib):
    p = W.frac_lap_1d(100)
    p["LW"] = 2.0 + 1e-3   # not a whole number of steps is only checked at build; plan ok
    with pytest.raises(hmat.HMError):
        hmat.plan_info(dict(p, dim=3), W.default_opts())
    with pytest.raises(hmat.HMError):
        hmat.plan_info(p, W.default_opts(leaf=0))
    with pytest.raises(hmat.HMError):
        hmat.plan_info(dict(p, s=1.5), W.default_opts())


def test_precision_and_solve_options_are_checked():
    """Mixed-precision storage exists for the hierarchical-inverse solve of 1D
    problems only: elsewhere (2D, or the substitution solve) it is an argument
    error, never a silent FP64 run; unknown modes and bad tolerances too."""
    p1 = W.frac_lap_1d(255, 0.5)
    p2 = W.frac_lap_2d(16, 0.5)
    for prec in ("mixed_fp32", "mixed_bf16"):
        hmat.plan_info(p1, W.default_opts(leaf=32, precision=prec))
        hmat.plan_info(p1, W.default_opts(leaf=32, precision=prec, solve="hinv"))
        with pytest.raises(hmat.HMError):
            hmat.plan_info(p1, W.default_opts(leaf=32, precision=prec, solve="subst"))
        with pytest.raises(hmat.HMError):
            hmat.plan_info(p2, W.default_opts(leaf=32, precision=prec))
    with pytest.raises(hmat.HMError):
        hmat.plan_info(p2, W.default_opts(leaf=32, solve="hinv"))
    with pytest.raises(hmat.HMError):
        hmat.plan_info(p1, W.default_opts(leaf=2048, solve="hinv"))
    with pytest.raises(hmat.HMError):
        hmat.plan_info(p1, W.default_opts(leaf=32, precision=7))
    with pytest.raises(hmat.HMError):
        hmat.plan_info(p1, W.default_opts(leaf=32, solve=9))
    with pytest.raises(hmat.HMError):
        hmat.plan_info(p1, W.default_opts(leaf=32, hinv_tol=1.5))
    with pytest.raises(hmat.HMError):
        hmat.plan_info(p1, W.default_opts(leaf=32, solve_block=-1))
    for form in ("identity", "literal"):
        hmat.plan_info(p1, W.default_opts(leaf=32, cn_form=form))
    with pytest.raises(hmat.HMError):
        hmat.plan_info(p1, W.default_opts(leaf=32, cn_form=2))


def test_solve_block_option_changes_the_substitution_plan():
    """opts.solve_block sets the rows of the substitution solve's blocks: at
    N = 4095 the default (1024-row blocks) and 2048-row blocks give different
    schedules, and the larger blocks need fewer dependency waves."""
    p = W.levy_1d(4095)
    o = W.default_opts(leaf=128, max_rank=32, lu_max_rank=16, solve="subst")
    a = hmat.plan_factor(p, o)
    b = hmat.plan_factor(p, dict(o, solve_block=2048))
    assert a["bad_spans"] == 0 and b["bad_spans"] == 0
    assert b["solve_waves"] < a["solve_waves"]
    assert b["gemm_fma"][1] > a["gemm_fma"][1]  # larger dense inverses of the solve blocks


def test_splitmix64_published_outputs_and_batch_stream():
    """splitmix64 with seed 0 gives the reference implementation's first
    outputs; the batched workload's parameters stay in their ranges."""
    g = W.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    batch = W.levy_batch(512)
    ns = np.array([p["n"][0] for p, _ in batch])
    assert ns.min() >= 1024 and ns.max() <= 32768
    assert 4.0e6 < ns.sum() < 5.2e6
    for p, o in batch[:32]:
        assert 0.25 <= p["s"] <= 0.95 and -1 <= p["b"][0] <= 1 and 0 <= p["a"] <= 0.125
    assert W.levy_batch(4) == W.levy_batch(4)


@pytest.mark.parametrize("case", ["levy1d", "frac2d", "lshape"])
def test_streamed_planning_matches_one_piece(case, monkeypatch):
    """The H-LU plan handed out in slices (as the factorisation streams it to
    the executor) and merged in groups of consecutive slices gives every op
    exactly the producers of the one-piece plan that lie in its group, in the
    same wave order (host self-check of the dry run; any mismatch is an error)."""
    if case == "levy1d":
        prob, opts, dt, steps, kind = W.WORKLOADS["levy_1d_n65536"]
        opts, theta = dict(opts, lu_max_rank=16, lu_tol=1e-10), -0.5 * dt
    elif case == "frac2d":
        prob = W.frac_lap_2d(64)
        opts, theta = W.default_opts(leaf=64, aca_tol=1e-8, max_rank=25, lu_tol=1e-8, lu_max_rank=25), -1e-3
    else:
        prob, opts, theta = W.lshape_poisson(47), W.default_opts(leaf=64, max_rank=32, lu_max_rank=32), 1.0
    monkeypatch.setenv("HM_CHECK_STREAM", "777")
    info = hmat.plan_factor(prob, opts, theta)
    assert info["fact_ops"] > 777 * 8


def test_injected_allocation_failure_is_reported_and_never_streamed(monkeypatch):
    """Host-side fault injection: the dry run's allocations fail past
    HM_ARENA_LIMIT_BYTES as a full device would.  Planning reports
    HM_ERR_OOM, and the streamed planning hands out no slice with an operand
    outside the allocations that succeeded (checked under HM_CHECK_STREAM;
    a violation would be reported as HM_ERR_ARG instead)."""
    prob, opts, dt, steps, kind = W.WORKLOADS["levy_1d_n65536"]
    opts = dict(opts, lu_max_rank=16, lu_tol=1e-10)
    monkeypatch.setenv("HM_ARENA_LIMIT_BYTES", str(2 * 10 ** 9))
    with pytest.raises(hmat.HMError) as e:
        hmat.plan_factor(prob, opts, -0.5 * dt)
    assert e.value.status == -2
    monkeypatch.setenv("HM_CHECK_STREAM", "777")
    with pytest.raises(hmat.HMError) as e:
        hmat.plan_factor(prob, opts, -0.5 * dt)
    assert e.value.status == -2, str(e.value)
    monkeypatch.setenv("HM_ARENA_LIMIT_BYTES", str(10 ** 12))   # room enough: plans
    assert hmat.plan_factor(prob, opts, -0.5 * dt)["fact_ops"] > 0


def test_autotune_search_space_per_precision_and_dimension():
    """The autotuner's candidates (no GPU): a 1D box problem gets the inverses
    and the substitution solve at every block below N; a mixed precision keeps
    only the inverses (its refinement needs them); a 2D problem gets only the
    substitution solve, and a 2D problem in a mixed precision has no candidate
    at all, which is an error rather than an empty choice."""
    from paper_1812_08324_gb300 import autotune
    p1, o1 = W.levy_batch(1)[0]
    n1 = p1["n"][0]
    c64 = autotune.configurations(p1, o1, leafs=(64,), solve_blocks=(256, 1 << 30))
    assert {(c["solve"], c.get("solve_block", 0)) for c in c64} == {("hinv", 0), ("subst", 256)}
    mixed = autotune.configurations(p1, dict(o1, precision="mixed_fp32"), leafs=(32, 64))
    assert mixed and all(c["solve"] == "hinv" for c in mixed)
    assert {c["leaf"] for c in mixed} == {32, 64}
    assert all(c["leaf"] <= n1 for c in autotune.configurations(p1, o1, leafs=(64, 1 << 20)))
    p2 = W.frac_lap_2d(64, 0.5)
    c2 = autotune.configurations(p2, W.default_opts(leaf=64), leafs=(64,), solve_blocks=(1024,))
    assert c2 == [{"leaf": 64, "solve": "subst", "solve_block": 1024}]
    with pytest.raises(ValueError):
        autotune.configurations(p2, W.default_opts(leaf=64, precision="mixed_fp32"), leafs=(64,))


def test_plan_histogram_counts_every_op(monkeypatch, capfd):
    """HM_PLAN_HIST=1 prints the planned H-LU's tasks by op kind; the op
    counts it reports add up to the dry run's fact_ops, and the GEMM task
    count is at least the GEMM op count (one or more 32 x 32 tiles each)."""
    prob, opts, dt, steps, kind = W.WORKLOADS["frac_lap_1d_n1023"]
    monkeypatch.setenv("HM_PLAN_HIST", "1")
    info = hmat.plan_factor(prob, dict(opts, lu_max_rank=16, max_rank=16), -0.5 * dt)
    err = capfd.readouterr().err
    rows = {}
    for line in err.splitlines():
        m = re.match(r"\[plan\] (\w+)\s+(\d+) ops\s+(\d+) tasks", line)
        if m:
            rows[m.group(1)] = (int(m.group(2)), int(m.group(3)))
    assert set(rows) == {"gemm", "lu", "trunc", "copy", "reduce"}
    assert sum(o for o, _ in rows.values()) == info["fact_ops"]
    assert rows["gemm"][1] >= rows["gemm"][0] > 0 and rows["lu"][0] > 0
