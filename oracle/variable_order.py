"""Dense FP64 CPU oracle for the variable-order fractional Poisson problem on
the L-shaped domain (Sec. "Application: Variable-Order Fractional Poisson
Equation").

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this module.  It shares no code with the CUDA path.

The problem: G u = f on Omega = [-1,1]^2 minus [0,1]^2 with u = 0 outside,
where G = -(-Delta)^{s(x)} is the generator whose row at x uses the order
s(x) = 0.9 - 0.8 d(x), d(x) the distance from x to the boundary of Omega, and
f(x) = sum_k exp(-10 |x - x_k|^2) with x_k = (-1/2, 1/2), (1/2, -1/2),
(-1/2, -1/2).

Discretisation: the interior grid of [-1,1]^2 (n points per axis, h = 2/(n+1))
restricted to Omega; row i of G is row i of the constant-order discrete
generator of ``levy_dense`` with s = s(x_i) (the singular discretisation of
Sec. "Singular and/or Slow Decaying Levy Measure"), restricted to the points
of Omega (u vanishes on the removed quadrant, which the jump sums then skip),
with the window L_W = 2 covering every pair of points.

Readings:
* The paper writes -(-Delta)^{s(x)} u = f; with G = -(-Delta)^s that is G u = f.
* Omega excludes the closed quadrant [0,1]^2: grid points with x >= 0 and
  y >= 0 are not unknowns.
* For a variable order the row at x_i uses the kernel, the window sums, the
  tail and the local diffusion coefficient of the order s(x_i) (the paper
  gives the discretisation only for constant s and applies it row by row).

Parity unpinned: nothing; see tests/test_oracle_variable_order.py.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import linalg

from . import levy_dense as LD

SOURCES = ((-0.5, 0.5), (0.5, -0.5), (-0.5, -0.5))


def lshape_problem(n: int, s_center: float = 0.9, s_slope: float = 0.8) -> dict:
    """The problem dict: n x n interior grid of [-1,1]^2 (h = 2/(n+1)),
    window L_W = 2 = (n+1) h, rho support r = 0.2, untruncated stable kernel."""
    return dict(dim=2, n=[n, n], lo=[-1.0, -1.0], hi=[1.0, 1.0], a=0.0, b=[0.0, 0.0], c=0.0,
                kernel=LD.STABLE, s=s_center, eps=0.0, lam=0.0, trunc=math.inf, LW=2.0, r=0.2,
                domain="L", s_slope=s_slope)


def inside_mask(prob: dict) -> np.ndarray:
    """Natural-order mask of the full grid: False on the removed closed
    quadrant x >= 0, y >= 0 (exact integer test: x_a = -1 + (i_a + 1) h >= 0
    iff 2 (i_a + 1) >= n + 1)."""
    n0, n1 = prob["n"]
    i1, i0 = np.divmod(np.arange(n0 * n1), n0)
    return ~((2 * (i0 + 1) >= n0 + 1) & (2 * (i1 + 1) >= n1 + 1))


def points(prob: dict) -> np.ndarray:
    """Coordinates of the unknowns, in natural order of the full grid with
    the removed points skipped."""
    return LD.grid_points(prob)[inside_mask(prob)]


def boundary_distance(X: np.ndarray) -> np.ndarray:
    """d(x): distance to the boundary of Omega = [-1,1]^2 minus [0,1]^2, the
    smaller of the distance to the outer square's sides and the distance to
    the removed quadrant."""
    X = np.asarray(X, dtype=np.float64)
    outer = np.minimum(1.0 - np.abs(X[:, 0]), 1.0 - np.abs(X[:, 1]))
    gx = np.maximum(0.0, -X[:, 0])
    gy = np.maximum(0.0, -X[:, 1])
    quad = np.sqrt(gx * gx + gy * gy)
    return np.minimum(outer, quad)


def order(prob: dict, X: np.ndarray) -> np.ndarray:
    """s(x) = s_center - s_slope d(x)."""
    return prob["s"] - prob["s_slope"] * boundary_distance(X)


def source(X: np.ndarray) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    f = np.zeros(X.shape[0])
    for c in SOURCES:
        f += np.exp(-10.0 * ((X[:, 0] - c[0]) ** 2 + (X[:, 1] - c[1]) ** 2))
    return f


def generator_rows(prob: dict, rows=None) -> np.ndarray:
    """Rows of the variable-order generator over the unknowns of Omega
    (all rows when ``rows`` is None).  Row i: the constant-order row with
    s = s(x_i) (levy_dense's Eq. Aij with the singular corrections), restricted
    to the columns of Omega."""
    mask = inside_mask(prob)
    idx_full = LD._grid_index(prob)
    nat = np.nonzero(mask)[0]
    X = LD.grid_points(prob)[mask]
    s_all = order(prob, X)
    rows = range(len(nat)) if rows is None else rows
    out = np.empty((len(list(rows)), len(nat)))
    cache = {}
    for r_out, i in enumerate(rows):
        si = float(s_all[i])
        p = dict(prob, s=si)
        if si not in cache:
            cache[si] = LD.jump_constants(p)
        full = LD._row(p, cache[si], idx_full, int(nat[i]))
        out[r_out] = full[mask]
    return out


def generator_dense(prob: dict) -> np.ndarray:
    return generator_rows(prob)


def poisson_solve(prob: dict) -> np.ndarray:
    """u with G u = f by dense LU with partial pivoting (LAPACK via scipy)."""
    G = generator_dense(prob)
    f = source(points(prob))
    return linalg.lu_solve(linalg.lu_factor(G, check_finite=False), f, check_finite=False)
