"""Synthetic workloads shaped like the paper's experiments.

This module only *describes* inputs: grid and kernel parameters, solver
options, initial data and the forcing of manufactured solutions.  It holds
none of the method's arithmetic (no generator entries, no H-matrix, no time
stepping) and is the one module that both the CUDA path's callers and the
dense oracle's tests read, so that both sides see the same inputs.

Every array is built from closed-form expressions of the grid coordinates;
random vectors come from a seeded ``numpy.random.Generator``.

Problem dictionaries use the field names of the C struct ``hm_problem``
(``include/levy_hmat.h``); option dictionaries those of ``hm_opts``.
"""
from __future__ import annotations

import math

import numpy as np

GAUSS = "gauss"
STABLE = "stable"


def frac_lap_const_k(d: int, s: float) -> float:
    """K_{d,s} = 4^s Gamma(1+s) Gamma(d/2+s) / Gamma(d/2): the value of
    (-Delta)^s (1-|x|^2)_+^s on the unit ball, used to manufacture forcing."""
    return 4.0 ** s * math.gamma(1.0 + s) * math.gamma(d / 2.0 + s) / math.gamma(d / 2.0)


def coords(prob: dict) -> np.ndarray:
    """Interior grid coordinates, natural order (axis 0 fastest), shape (N, dim)."""
    d = prob["dim"]
    h = (prob["hi"][0] - prob["lo"][0]) / (prob["n"][0] + 1)
    axes = [prob["lo"][a] + h * np.arange(1, prob["n"][a] + 1) for a in range(d)]
    if d == 1:
        return axes[0][:, None]
    X0, X1 = np.meshgrid(axes[0], axes[1], indexing="xy")
    return np.stack([X0.ravel(), X1.ravel()], axis=1)


# ----------------------------------------------------------------------------
# Workload 1: 1D fractional Laplacian s = 1/2, N = 1023, manufactured solution
# ----------------------------------------------------------------------------

def frac_lap_1d(n: int = 1023, s: float = 0.5) -> dict:
    """(-Delta)^s on [-1, 1] with u = 0 outside, h = 2/(n+1), L_W = 2, r = 0.2."""
    return dict(dim=1, n=[n, 1], lo=[-1.0, 0.0], hi=[1.0, 0.0], a=0.0, b=[0.0, 0.0], c=0.0,
                kernel=STABLE, s=s, eps=0.0, lam=0.0, trunc=math.inf, LW=2.0, r=0.2)


def manufactured_unit_ball(prob: dict):
    """u(x, t) = (1 - |x|^2)_+^s e^{-t}; with u_t = -(-Delta)^s u + f this needs
    f = (K_{d,s} - (1 - |x|^2)^s) e^{-t} inside the ball.  Returns (u0, f(t), u(t))."""
    X = coords(prob)
    s = prob["s"]
    prof = np.clip(1.0 - np.sum(X * X, axis=1), 0.0, None) ** s
    K = frac_lap_const_k(prob["dim"], s)
    return prof.copy(), (lambda t: (K - prof) * math.exp(-t)), (lambda t: prof * math.exp(-t))


# ----------------------------------------------------------------------------
# Workload 2: 1D full Levy generator, alpha-stable alpha = 1.5 truncated to |y| <= 2
# ----------------------------------------------------------------------------

def levy_1d(n: int = 65536, sigma: float = 0.2, b: float = 0.3, alpha: float = 1.5) -> dict:
    """Drift b, diffusion a = sigma^2/2, symmetric alpha-stable jumps
    nu = c_{1,alpha/2}/|y|^{1+alpha} on |y| <= 2, on [-1, 1] with h = 2/(n+1),
    so that L_W = 2 = (n+1) h and the truncation radius equals the window."""
    return dict(dim=1, n=[n, 1], lo=[-1.0, 0.0], hi=[1.0, 0.0], a=0.5 * sigma * sigma,
                b=[b, 0.0], c=0.0, kernel=STABLE, s=0.5 * alpha, eps=0.0, lam=0.0,
                trunc=2.0, LW=2.0, r=0.2)


def gaussian_u0(prob: dict, beta: float = 50.0, center=(0.0, 0.0)) -> np.ndarray:
    """u0 = exp(-beta |x - center|^2) (the paper's 1D initial data for beta = 50)."""
    X = coords(prob)
    c = np.asarray(center[: prob["dim"]])
    return np.exp(-beta * np.sum((X - c) ** 2, axis=1))


# ----------------------------------------------------------------------------
# Workload 3: 2D fractional Laplacian on the unit square, 256 x 256
# ----------------------------------------------------------------------------

def frac_lap_2d(n: int = 256, s: float = 0.75) -> dict:
    """(-Delta)^s on [0,1]^2 with u = 0 outside, h = 1/(n+1), square window
    L_W = 1 = (n+1) h (max-norm), r = 0.2."""
    return dict(dim=2, n=[n, n], lo=[0.0, 0.0], hi=[1.0, 1.0], a=0.0, b=[0.0, 0.0], c=0.0,
                kernel=STABLE, s=s, eps=0.0, lam=0.0, trunc=math.inf, LW=1.0, r=0.2)


def bump_u0(prob: dict, sigma: float = 0.1) -> np.ndarray:
    """Gaussian bump exp(-|x - (1/2, 1/2)|^2 / (2 sigma^2))."""
    return gaussian_u0(prob, beta=1.0 / (2.0 * sigma * sigma), center=(0.5, 0.5))


# ----------------------------------------------------------------------------
# Merton (Gaussian) jumps, the paper's timing workload
# ----------------------------------------------------------------------------

def merton_1d(n: int = 1023, eps2: float = 5.0, LW: float = 2.0) -> dict:
    """nu = exp(-5 y^2) on [-1, 1] (Eq. model1d), h = 2/(n+1)."""
    return dict(dim=1, n=[n, 1], lo=[-1.0, 0.0], hi=[1.0, 0.0], a=0.0, b=[0.0, 0.0], c=0.0,
                kernel=GAUSS, s=0.0, eps=math.sqrt(eps2), lam=1.0, trunc=math.inf, LW=LW, r=0.2)


# ----------------------------------------------------------------------------
# Variable-order fractional Poisson problem on the L-shaped domain
# (Sec. "Application: Variable-Order Fractional Poisson Equation")
# ----------------------------------------------------------------------------

LSHAPE_SOURCES = ((-0.5, 0.5), (0.5, -0.5), (-0.5, -0.5))


def lshape_poisson(n: int = 255, s_center: float = 0.9, s_slope: float = 0.8) -> dict:
    """G u = f on [-1,1]^2 minus [0,1]^2, u = 0 outside: the n x n interior grid
    of the square (h = 2/(n+1)) without the points of the closed upper-right
    quadrant, order s(x) = s_center - s_slope d(x) per row, window L_W = 2."""
    return dict(dim=2, n=[n, n], lo=[-1.0, -1.0], hi=[1.0, 1.0], a=0.0, b=[0.0, 0.0], c=0.0,
                kernel=STABLE, s=s_center, eps=0.0, lam=0.0, trunc=math.inf, LW=2.0, r=0.2,
                domain="L", s_slope=s_slope)


def lshape_coords(prob: dict) -> np.ndarray:
    """Coordinates of the unknowns of the L-shaped domain in natural order
    (the square's order with the removed points skipped)."""
    n0, n1 = prob["n"]
    i1, i0 = np.divmod(np.arange(n0 * n1), n0)
    keep = ~((2 * (i0 + 1) >= n0 + 1) & (2 * (i1 + 1) >= n1 + 1))
    return coords(prob)[keep]


def lshape_source(prob: dict) -> np.ndarray:
    """f(x) = sum of three Gaussians exp(-10 |x - x_k|^2) at the unknowns."""
    X = lshape_coords(prob)
    f = np.zeros(X.shape[0])
    for cx, cy in LSHAPE_SOURCES:
        f += np.exp(-10.0 * ((X[:, 0] - cx) ** 2 + (X[:, 1] - cy) ** 2))
    return f


def default_opts(**kw) -> dict:
    o = dict(leaf=64, eta=1.0, aca_tol=1e-10, max_rank=64, lu_tol=1e-10, lu_max_rank=64,
             precision="fp64", refine_tol=1e-13, refine_max=4)
    o.update(kw)
    return o


WORKLOADS = {
    # name: (problem, options, dt, steps, initial-data kind)
    "frac_lap_1d_n1023": (frac_lap_1d(1023, 0.5), default_opts(leaf=64, aca_tol=1e-10, max_rank=64),
                          1e-3, 100, "unit_ball"),
    "levy_1d_n65536": (levy_1d(65536), default_opts(leaf=256, aca_tol=1e-10, max_rank=32),
                       1e-3, 1000, "gauss50"),
    "frac_lap_2d_256x256_s0.75": (frac_lap_2d(256, 0.75), default_opts(leaf=256, aca_tol=1e-8, max_rank=64),
                                  1.0 / 200, 200, "bump"),
    "frac_lap_2d_256x256_s0.3": (frac_lap_2d(256, 0.3), default_opts(leaf=256, aca_tol=1e-8, max_rank=64),
                                 1.0 / 200, 200, "bump"),
}


# ----------------------------------------------------------------------------
# Workload 4: many independent 1D Levy solves (batched), parameters drawn by
# splitmix64 (seed 0) in the order N, alpha, b, sigma per solve
# ----------------------------------------------------------------------------

_M64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then
    two xor-shift-multiply rounds; uniform doubles from the top 53 bits."""

    def __init__(self, seed: int = 0):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        return a + (b - a) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def batch_leaf(n: int) -> int:
    """Leaf size of a batched solve by problem size (the rule the leaf autotuner
    starts from; see autotune.py)."""
    return 256 if n >= 8192 else (128 if n >= 2048 else 64)


def levy_batch(count: int = 512, seed: int = 0, log2_lo: float = 10.0, log2_hi: float = 15.0):
    """The batched workload: per solve N = round(2^U(10,15)), alpha ~ U(0.5,1.9),
    b ~ U(-1,1), sigma ~ U(0,0.5); truncation 2, u0 = exp(-50 x^2),
    dt = 1/500, 500 steps; ACA rank <= 32, factor rank <= 16.  Returns a list
    of (problem, options); dt and steps are LEVY_BATCH_DT / LEVY_BATCH_STEPS."""
    g = SplitMix64(seed)
    out = []
    for _ in range(count):
        n = int(round(2.0 ** g.uniform(log2_lo, log2_hi)))
        alpha = g.uniform(0.5, 1.9)
        b = g.uniform(-1.0, 1.0)
        sigma = g.uniform(0.0, 0.5)
        prob = levy_1d(n, sigma=sigma, b=b, alpha=alpha)
        opts = default_opts(leaf=batch_leaf(n), aca_tol=1e-10, max_rank=32, lu_tol=1e-10, lu_max_rank=16,
                            refine_max=0)
        out.append((prob, opts))
    return out


LEVY_BATCH_DT = 1.0 / 500
LEVY_BATCH_STEPS = 500


# ----------------------------------------------------------------------------
# Workload 5: a served request stream (Poisson arrivals, splitmix64 seed 0)
# ----------------------------------------------------------------------------

def serve_stream(count: int = 2000, seed: int = 0, rate: float = 200.0, log2_1d=(10.0, 16.0),
                 sides_2d=(64, 128, 256, 512), steps=(100, 1000)):
    """Requests in arrival order, drawn per request in this order: the
    exponential inter-arrival gap (rate per second), 1D or 2D (half each),
    N = round(2^U(log2_1d)) or a side from sides_2d, s ~ U(0.2, 0.9), steps
    ~ U{steps}; dt = 1/steps.  Fractional Laplacian with a Gaussian bump.
    Returns dicts with arrival (s), problem, opts, dt, steps, u0."""
    g = SplitMix64(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += -math.log(max(g.uniform(), 1e-300)) / rate
        two_d = g.uniform() >= 0.5
        if two_d:
            side = int(sides_2d[min(int(g.uniform() * len(sides_2d)), len(sides_2d) - 1)])
        else:
            n = int(round(2.0 ** g.uniform(*log2_1d)))
        s = g.uniform(0.2, 0.9)
        st = steps[0] + min(int(g.uniform() * (steps[1] - steps[0] + 1)), steps[1] - steps[0])
        if two_d:
            prob = frac_lap_2d(side, s)
            opts = default_opts(leaf=256, aca_tol=1e-8, max_rank=64, lu_tol=1e-10, lu_max_rank=16, refine_max=0)
            u0 = bump_u0(prob)
        else:
            prob = frac_lap_1d(n, s)
            opts = default_opts(leaf=batch_leaf(n), aca_tol=1e-10, max_rank=32, lu_tol=1e-10, lu_max_rank=16,
                                refine_max=0)
            u0 = gaussian_u0(prob, 50.0)
        out.append(dict(rid=rid, arrival=t, problem=prob, opts=opts, dt=1.0 / st, steps=st, u0=u0))
    return out


def initial_data(prob: dict, kind: str) -> np.ndarray:
    if kind == "unit_ball":
        return manufactured_unit_ball(prob)[0]
    if kind == "gauss50":
        return gaussian_u0(prob, 50.0)
    if kind == "bump":
        return bump_u0(prob)
    raise ValueError(kind)


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal test vector."""
    return np.random.default_rng(seed).standard_normal(n)
