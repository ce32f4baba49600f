"""Pins of the variable-order L-shaped oracle (Sec. "Application: Variable-
Order Fractional Poisson Equation") against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle import levy_dense as LD
from oracle import variable_order as VO


def test_boundary_distance_closed_values():
    X = np.array([[-0.5, 0.5], [-0.5, -0.5], [-0.1, 0.9], [0.7, -0.2], [-0.9, -0.3], [-0.25, -0.25]])
    d = VO.boundary_distance(X)
    # (-0.5, 0.5): 0.5 to x = -1 and to x = 0; (-0.5,-0.5): 0.5 to the outer sides;
    # (-0.1, 0.9): 0.1 to y = 1 and to x = 0; (0.7,-0.2): 0.2 to y = 0 (quadrant);
    # (-0.9,-0.3): 0.1 to x = -1; (-0.25,-0.25): sqrt(2)/4 to the quadrant's corner
    np.testing.assert_allclose(d, [0.5, 0.5, 0.1, 0.2, 0.1, math.sqrt(2) / 4], rtol=0, atol=1e-15)


def test_order_range_and_mask():
    prob = VO.lshape_problem(31)
    X = VO.points(prob)
    assert X.shape[0] == 31 * 31 - 16 * 16                      # 16 x 16 points have x, y >= 0
    assert not np.any((X[:, 0] >= 0) & (X[:, 1] >= 0))
    s = VO.order(prob, X)
    # the largest distance to the boundary is on the diagonal x = y = -t where
    # 1 - t = sqrt(2) t: d_max = sqrt(2) / (1 + sqrt(2))
    dmax = math.sqrt(2) / (1 + math.sqrt(2))
    assert VO.boundary_distance(np.array([[-1 / (1 + math.sqrt(2))] * 2]))[0] == pytest.approx(dmax)
    assert s.min() >= 0.9 - 0.8 * dmax - 1e-12 and s.max() < 0.9 and np.all((s > 0) & (s < 1))


def test_constant_order_is_the_principal_submatrix():
    """s_slope = 0: the L-shaped generator is the square's generator (pinned in
    test_oracle_pins.py) restricted to Omega's rows and columns; symmetric."""
    prob = VO.lshape_problem(15, s_center=0.6, s_slope=0.0)
    G = VO.generator_dense(prob)
    sq = dict(prob)
    sq.pop("domain")
    Gs = LD.generator_dense(sq)
    m = VO.inside_mask(prob)
    np.testing.assert_allclose(G, Gs[np.ix_(m, m)], rtol=1e-14, atol=0)
    np.testing.assert_allclose(G, G.T, rtol=1e-12, atol=0)


def test_rows_reproduce_the_ball_closed_form_per_order():
    """(-Delta)^s (rho^2 - |x - c|^2)_+^s = K_{2,s} for any radius rho (scaling
    of the unit-ball closed form).  Row i (order s_i) applied to the profile
    with exponent s_i, for rows well inside the ball of radius 1/2 around
    (-1/2,-1/2) (inside Omega), approaches -K_{2,s_i}."""
    prob = VO.lshape_problem(47)
    X = VO.points(prob)
    c = np.array([-0.5, -0.5])
    s_all = VO.order(prob, X)
    r2 = np.sum((X - c) ** 2, axis=1)
    rows = np.nonzero(r2 < 0.15 ** 2)[0][:6]
    G = VO.generator_rows(prob, rows)
    errs = []
    for k, i in enumerate(rows):
        u = np.maximum(0.25 - r2, 0.0) ** s_all[i]
        errs.append(abs(G[k] @ u + LD.k_ds(2, s_all[i])) / LD.k_ds(2, s_all[i]))
    assert max(errs) < 5e-3, errs   # discretisation error ~1e-3; a wrong order misses by > 50%


def test_solution_is_symmetric_under_axis_swap():
    """Omega, s(x) and f are invariant under (x, y) -> (y, x), so the discrete
    solution is too (the grid maps onto itself)."""
    n = 23
    prob = VO.lshape_problem(n)
    u = VO.poisson_solve(prob)
    X = VO.points(prob)
    key = {(round(a, 12), round(b, 12)): k for k, (a, b) in enumerate(X)}
    swap = np.array([key[(round(b, 12), round(a, 12))] for a, b in X])
    np.testing.assert_allclose(u, u[swap], rtol=1e-10, atol=1e-14)
    assert np.all(u < 0)   # G = -(-Delta)^s: positive sources give a negative solution


def test_per_order_constants_are_smooth_in_s():
    """The per-row constants lambda_W(s), T(s), kappa(s) of the variable-order
    rows are analytic in s over the range the L-shaped problem uses: a
    24-node Chebyshev interpolant (what the device evaluates per row)
    reproduces the oracle's direct evaluation to 1e-12 of their scale."""
    prob = VO.lshape_problem(127)
    s = VO.order(prob, VO.points(prob))
    lo, hi = float(s.min()), float(s.max())
    M = 24
    t = np.cos(np.pi * (np.arange(M) + 0.5) / M)
    nodes = 0.5 * (lo + hi) + 0.5 * (hi - lo) * t
    F = np.array([LD.jump_constants(dict(prob, s=float(x))) for x in nodes])   # M x 3
    k = np.arange(M)
    C = (2.0 / M) * np.cos(np.outer(k, np.pi * (np.arange(M) + 0.5) / M)) @ F
    C[0] *= 0.5
    probe = np.random.default_rng(1).uniform(lo, hi, 12)
    for x in probe:
        tt = (x - 0.5 * (lo + hi)) / (0.5 * (hi - lo))
        approx = np.polynomial.chebyshev.chebval(tt, C)
        exact = np.array(LD.jump_constants(dict(prob, s=float(x))))
        scale = np.abs(F).max(axis=0)
        assert np.all(np.abs(approx - exact) <= 1e-12 * scale), (x, approx, exact)
