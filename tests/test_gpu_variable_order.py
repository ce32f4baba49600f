"""GPU parity of the variable-order fractional Poisson problem on the L-shaped
domain (Sec. "Application: Variable-Order Fractional Poisson Equation")
against the dense FP64 oracle: generator entries, the compressed H-matrix,
the H-matvec, H-LU of G itself and the preconditioned Poisson solve."""
import numpy as np
import pytest

from oracle import variable_order as V
from paper_1812_08324_gb300 import hmat, workloads as W

from gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu

# (n, leaf): n = 31 gives 705 unknowns, n = 47 gives 1633 (several tree levels
# and leaves cut by the removed quadrant)
CASES = [(31, 64), (47, 64), (48, 100)]


def _opts(leaf):
    return W.default_opts(leaf=leaf, aca_tol=1e-11, max_rank=48, lu_tol=1e-11, lu_max_rank=48)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def dense():
    cache = {}

    def get(n):
        if n not in cache:
            prob = V.lshape_problem(n)
            cache[n] = (prob, V.generator_dense(prob), V.poisson_solve(prob))
        return cache[n]
    return get


@pytest.mark.parametrize("n,leaf", CASES)
def test_entries_match_oracle(n, leaf, dense):
    """Every generator entry from the device formula equals the oracle's row
    of order s(x_i).  The per-row constants (window sums, tail, diffusion
    coefficient) come from a 24-node Chebyshev interpolant in s on the device
    and from direct evaluation in the oracle: 1e-11 of the row's diagonal."""
    prob, G, _ = dense(n)
    N = G.shape[0]
    H = hmat.HMatrix(W.lshape_poisson(n), _opts(leaf))
    assert H.n == N
    rows, cols = np.divmod(np.arange(N * N), N)
    got = host(H.entries(torch.from_numpy(rows), torch.from_numpy(cols))).reshape(N, N)
    scale = np.abs(np.diag(G))[:, None]
    err = np.max(np.abs(got - G) / scale)
    assert err < 1e-11, err
    H.free()


@pytest.mark.parametrize("n,leaf", CASES)
def test_hmatrix_and_matvec_match_dense(n, leaf, dense):
    """The compressed matrix and the H-matvec agree with the dense generator
    to the ACA tolerance."""
    prob, G, _ = dense(n)
    H = hmat.HMatrix(W.lshape_poisson(n), _opts(leaf))
    D = host(H.to_dense())
    assert np.linalg.norm(D - G) / np.linalg.norm(G) < 1e-9
    x = np.random.default_rng(3).standard_normal(G.shape[0])
    y = host(H.matvec(dev(x)))
    ref = G @ x
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-9
    H.free()


@pytest.mark.parametrize("n,leaf", CASES)
def test_poisson_solve_matches_oracle(n, leaf, dense):
    """H-LU of G (alpha = 0, theta = 1) preconditions Richardson iteration to
    the dense LU solution of G u = f."""
    prob, G, u_ref = dense(n)
    H = hmat.HMatrix(W.lshape_poisson(n), _opts(leaf))
    F = H.factor_shifted(0.0, 1.0)
    f = W.lshape_source(W.lshape_poisson(n))
    u, iters, res = hmat.shifted_solve(H, F, dev(f), tol=1e-13, maxit=30)
    u = host(u)
    assert res <= 1e-13 and iters <= 10, (iters, res)
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < 1e-9, err
    # the H-LU alone is already a close inverse
    u0 = host(F.solve(dev(f)))
    assert np.linalg.norm(u0 - u_ref) / np.linalg.norm(u_ref) < 1e-6
    F.free()
    H.free()


@pytest.mark.parametrize("n,leaf", CASES[1:])
def test_coarse_preconditioner(n, leaf, dense):
    """The paper's setting: the operator compressed accurately, the
    preconditioner the H-LU of a 1e-4 compression (eps_1 = 1e-4, eps_2 =
    1e-10).  Richardson still reaches the dense solution; a preconditioner
    from another grid is refused."""
    prob, G, u_ref = dense(n)
    Hop = hmat.HMatrix(W.lshape_poisson(n), _opts(leaf))
    Hpre = hmat.HMatrix(W.lshape_poisson(n), W.default_opts(leaf=leaf, aca_tol=1e-4, max_rank=48, lu_tol=1e-10,
                                                            lu_max_rank=48))
    assert Hpre.stats()["max_rank_seen"] < Hop.stats()["max_rank_seen"]
    F = Hpre.factor_shifted(0.0, 1.0)
    f = W.lshape_source(W.lshape_poisson(n))
    u, iters, res = hmat.shifted_solve(Hop, F, dev(f), tol=1e-12, maxit=60)
    assert res <= 1e-12 and 1 <= iters <= 40, (iters, res)
    assert np.linalg.norm(host(u) - u_ref) / np.linalg.norm(u_ref) < 1e-9
    other = hmat.HMatrix(W.lshape_poisson(n - 2), _opts(leaf))
    with pytest.raises(hmat.HMError):
        hmat.shifted_solve(other, F, dev(np.ones(other.n)))
    for X in (F, other, Hpre, Hop):
        X.free()


def test_shifted_solve_of_cn_matrix():
    """hm_shifted_solve with hm_factor's factors solves I - dt/2 G (alpha = 1)."""
    n = 31
    prob = W.lshape_poisson(n)
    G = V.generator_dense(V.lshape_problem(n))
    dt = 1e-2
    H = hmat.HMatrix(prob, _opts(64))
    F = H.factor(-0.5 * dt)
    b = np.random.default_rng(5).standard_normal(G.shape[0])
    x, iters, res = hmat.shifted_solve(H, F, dev(b), tol=1e-13, maxit=20)
    ref = np.linalg.solve(np.eye(G.shape[0]) - 0.5 * dt * G, b)
    assert np.linalg.norm(host(x) - ref) / np.linalg.norm(ref) < 1e-11
    F.free()
    H.free()


def test_shifted_factors_refused_by_cn():
    prob = W.lshape_poisson(31)
    H = hmat.HMatrix(prob, _opts(64))
    F = H.factor_shifted(0.0, 1.0)
    u = dev(np.zeros(H.n))
    with pytest.raises(hmat.HMError):
        hmat.cn_step(H, F, 1e-2, u)
    with pytest.raises(hmat.HMError):
        hmat.cn_solve(H, F, 1e-2, 3, u)
    F.free()
    H.free()


def test_not_converged_is_reported():
    """maxit = 0 leaves the H-LU solve alone; a tolerance below it is reported
    as not converged, with the iterate and residual still returned."""
    prob = W.lshape_poisson(31)
    H = hmat.HMatrix(prob, W.default_opts(leaf=64, aca_tol=1e-6, max_rank=8, lu_tol=1e-4, lu_max_rank=8))
    F = H.factor_shifted(0.0, 1.0)
    f = dev(W.lshape_source(prob))
    with pytest.raises(hmat.HMError):
        hmat.shifted_solve(H, F, f, tol=1e-15, maxit=0)
    u, iters, res = hmat.shifted_solve(H, F, f, tol=1e-15, maxit=0, check=False)
    assert iters == 0 and 0.0 < res < 1.0
    F.free()
    H.free()


def test_full_size_sampled_residual():
    """n = 255 (48641 unknowns, the size of the paper's L-shaped runs' finer
    grids): residuals f_i - G_i u of the GPU solution on sampled rows of the
    exact generator (oracle rows), relative to sum_j |G_ij u_j|."""
    n = 255
    prob = W.lshape_poisson(n)
    H = hmat.HMatrix(prob, W.default_opts(leaf=256, aca_tol=1e-10, max_rank=48, lu_tol=1e-6,
                                          lu_max_rank=32))
    F = H.factor_shifted(0.0, 1.0)
    f = W.lshape_source(prob)
    u, iters, res = hmat.shifted_solve(H, F, dev(f), tol=1e-12, maxit=50)
    u = host(u)
    assert res <= 1e-12, (iters, res)
    rows = np.random.default_rng(7).choice(H.n, 48, replace=False)
    rows = np.concatenate([rows, [0, H.n - 1]])
    Gr = V.generator_rows(V.lshape_problem(n), rows)
    r = f[rows] - Gr @ u
    scale = np.abs(Gr) @ np.abs(u)
    assert np.max(np.abs(r) / scale) < 1e-8
    F.free()
    H.free()
