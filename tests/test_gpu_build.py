"""GPU parity of construction and H-matvec against the dense FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import levy_dense as O
from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu

SMALL = [
    ("frac1d", W.frac_lap_1d(1023, 0.5), W.default_opts(leaf=64, aca_tol=1e-10, max_rank=64)),
    ("levy1d", W.levy_1d(2047), W.default_opts(leaf=128, aca_tol=1e-10, max_rank=32)),
    ("merton1d", W.merton_1d(1000), W.default_opts(leaf=50, aca_tol=1e-10, max_rank=40)),
    ("frac2d", W.frac_lap_2d(40, 0.75), W.default_opts(leaf=64, aca_tol=1e-8, max_rank=64)),
    ("frac2d_s03", W.frac_lap_2d(33, 0.3), W.default_opts(leaf=50, aca_tol=1e-8, max_rank=64)),
    ("levy2d_drift", dict(W.frac_lap_2d(32, 0.6), a=0.01, b=[0.4, -0.2], c=-0.3, trunc=0.5),
     W.default_opts(leaf=64, aca_tol=1e-9, max_rank=64)),
]


def _stencil_mask(prob):
    """Diagonal and axis-neighbour pairs (natural order)."""
    n0 = prob["n"][0]
    N = n0 if prob["dim"] == 1 else n0 * prob["n"][1]
    idx = np.arange(N)
    if prob["dim"] == 1:
        d = np.abs(idx[:, None] - idx[None, :])
        return d <= 1
    i0, i1 = idx % n0, idx // n0
    d = np.abs(i0[:, None] - i0[None, :]) + np.abs(i1[:, None] - i1[None, :])
    return d <= 1


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def dense_cache():
    return {}


def oracle_G(name, prob, cache):
    if name not in cache:
        cache[name] = O.generator_dense(prob)
    return cache[name]


@pytest.mark.parametrize("name,prob,opts", SMALL, ids=[c[0] for c in SMALL])
def test_entries_match_oracle(name, prob, opts, dense_cache):
    """Every entry of G from the device generator equals the oracle's to a few ulps."""
    G = oracle_G(name, prob, dense_cache)
    H = hmat.HMatrix(prob, opts)
    N = G.shape[0]
    r, c = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    out = host(H.entries(torch.tensor(r.ravel()), torch.tensor(c.ravel()))).reshape(N, N)
    H.sync()
    near = _stencil_mask(prob)
    far = ~near
    assert np.all(np.abs(out[far] - G[far]) <= 4e-15 * np.abs(G[far]) + 1e-300)
    # the diagonal and the axis neighbours carry kappa = (moment - window sum)/(2h^2),
    # whose cancellation is exact only up to the summation order of the window sum
    gd = np.abs(np.diag(G))[:, None] * np.ones((1, N))
    assert np.all(np.abs(out[near] - G[near]) <= 1e-13 * gd[near])


@pytest.mark.parametrize("name,prob,opts", SMALL, ids=[c[0] for c in SMALL])
def test_hmatrix_blocks(name, prob, opts, dense_cache):
    """Dense leaves are exact; every ACA block meets ||B - U V'||_F <= c tol ||B||_F
    (brute force over the block)."""
    G = oracle_G(name, prob, dense_cache)
    H = hmat.HMatrix(prob, opts)
    D = host(H.to_dense())
    row0, m, col0, nc, typ, perm = hmat.plan_blocks(prob, opts)
    Gm = G[np.ix_(perm, perm)]
    Dm = D[np.ix_(perm, perm)]
    tol = opts["aca_tol"]
    st = H.stats()
    for b in range(len(row0)):
        sl = (slice(row0[b], row0[b] + m[b]), slice(col0[b], col0[b] + nc[b]))
        B, A = Gm[sl], Dm[sl]
        if typ[b] == 2:
            assert np.max(np.abs(A - B)) <= 1e-13 * np.max(np.abs(B))
        else:
            nb = np.linalg.norm(B)
            if st["rank_capped_blocks"] == 0:
                assert np.linalg.norm(A - B) <= 20 * tol * nb + 1e-300, (b, np.linalg.norm(A - B) / nb)
            else:
                assert np.linalg.norm(A - B) <= 1e-4 * nb


@pytest.mark.parametrize("name,prob,opts", SMALL, ids=[c[0] for c in SMALL])
def test_matvec_matches_dense(name, prob, opts, dense_cache):
    G = oracle_G(name, prob, dense_cache)
    H = hmat.HMatrix(prob, opts)
    N = G.shape[0]
    rng = np.random.default_rng(7)
    x, w1, w2 = rng.standard_normal(N), rng.standard_normal(N), rng.standard_normal(N)
    alpha, beta, gamma = 0.7, -1.3e-3, 0.25
    y = host(H.matvec(dev(x), alpha=alpha, beta=beta, gamma=gamma, w1=dev(w1), w2=dev(w2)))
    ref = alpha * x + beta * (G @ x) + gamma * (w1 + w2)
    # the H error is relative to |G| |x| (ACA error of the far field)
    scale = np.abs(beta) * (np.abs(G) @ np.abs(x)) + np.abs(ref)
    assert np.max(np.abs(y - ref) / scale) < 50 * opts["aca_tol"]
    # pure G x (beta = 1) too, smooth input
    xs = W.gaussian_u0(prob, 20.0)
    gx = host(H.matvec(dev(xs)))
    assert np.linalg.norm(gx - G @ xs) <= 50 * opts["aca_tol"] * np.linalg.norm(np.abs(G) @ np.abs(xs))
    H.sync()


def test_levy_65536_sampled_entries_and_stats():
    """Full-size 1D workload: build, sampled entries against the oracle's row
    formula, and the matvec of the smooth initial data against sampled dense rows."""
    prob, opts, dt, steps, kind = W.WORKLOADS["levy_1d_n65536"]
    H = hmat.HMatrix(prob, opts)
    st = H.stats()
    assert st["dense_blocks"] == 766 and st["lowrank_blocks"] == 1482
    rng = np.random.default_rng(3)
    rows = rng.integers(0, 65536, 24)
    u0 = W.initial_data(prob, kind)
    gx = host(H.matvec(dev(u0)))
    for i in rows:
        row = O.generator_dense_row(prob, int(i))
        got = host(H.entries(torch.tensor([int(i)] * 65536), torch.arange(65536)))
        far = np.abs(np.arange(65536) - i) > 1
        assert np.all(np.abs(got[far] - row[far]) <= 4e-15 * np.abs(row[far]) + 1e-300)
        assert np.all(np.abs(got[~far] - row[~far]) <= 1e-13 * abs(row[i]))
        ref = row @ u0
        assert abs(gx[i] - ref) <= 1e-8 * (np.abs(row) @ np.abs(u0))
    H.sync()
