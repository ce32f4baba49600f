"""Dense FP64 CPU oracle for the Crank-Nicolson scheme of a Levy generator.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this module.  It shares no code with the CUDA path: every formula below is
written out again, slowly and literally, from the paper (Xu & Darve,
"Efficient Numerical Method for Models Driven by Levy Process via Hierarchical
Matrices", arXiv 1812.08324).

What it computes (the plain definition the H-matrix method approximates):

* the dense discretised generator ``G`` (``G = -A`` in the paper's notation,
  Sec. "Numerical Scheme", Eq. (Aij)), including the singularity-subtraction
  discretisation of Sec. "Singular and/or Slow Decaying Levy Measure"
  (Eqs. I1approx, I2approx, I3approx) for kernels that blow up at the origin;
* Crank-Nicolson steps ``(I - dt/2 G) u^{n+1} = (I + dt/2 G) u^n
  + dt/2 (f^n + f^{n+1})`` (Eq. scheme) with a dense LU with partial pivoting
  (LAPACK through scipy, a library primitive).

Readings of the paper that this file relies on:

* G is the generator a d^2 + b d_2x + c + delta_L, i.e. minus the paper's A.
* Off-diagonal jump entries are w * nu(x_k - x_i) with trapezoid weight w
  (Eq. dl); lambda_W sums nu * w over *all* window offsets, including those
  whose target lies outside the grid (u = 0 there, the killed process).
* Window L_W = N_W h with an integer N_W; trapezoid weights are halved on the
  window's faces (per axis in 2D, a square max-norm window).
* The tail term of Eq. I2approx is -u(x) T, T = mass of nu outside the window
  (and inside the truncation radius); the far field f_x^{L_W} is zero because
  u vanishes outside the domain.
* The local diffusion coefficient of Eq. I3approx is (1/2) int rho nu y_d^2,
  with rho(y) = (1 - (|y|/r)^4)^3 on |y| < r, which meets Eq. rho_condition.
  The first-derivative sum of Eq. I1approx vanishes for even rho and nu.

Parity unpinned: nothing in this file is unpinned; each function is checked
against closed forms, invariants or the paper's printed values by
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, linalg

GAUSS = "gauss"
STABLE = "stable"


def c_ds(d: int, s: float) -> float:
    """Normalising constant of the fractional Laplacian, c_{d,s} =
    4^s Gamma(d/2 + s) / (pi^{d/2} |Gamma(-s)|)  (Introduction, definition of
    (-Delta)^s; the 1D form is restated in Sec. "Singular and/or Slow Decaying
    Levy Measure")."""
    return 4.0 ** s * math.gamma(d / 2.0 + s) / (math.pi ** (d / 2.0) * abs(math.gamma(-s)))


def k_ds(d: int, s: float) -> float:
    """(-Delta)^s (1 - |x|^2)_+^s = K_{d,s} on the unit ball, with
    K_{d,s} = 4^s Gamma(1+s) Gamma(d/2+s) / Gamma(d/2) (Sec. "Singular and Slow
    Decaying Levy Measure", the 1D fractional Poisson and 2D unit-ball examples)."""
    return 4.0 ** s * math.gamma(1.0 + s) * math.gamma(d / 2.0 + s) / math.gamma(d / 2.0)


# ----------------------------------------------------------------------------
# Problem description (a plain dict; keys mirror the C-ABI's hm_problem)
# ----------------------------------------------------------------------------

def _get(prob: dict, key, default):
    return prob[key] if key in prob else default


def spacing(prob: dict) -> float:
    """Uniform interior grid: n points per axis strictly inside [lo, hi],
    h = (hi - lo) / (n + 1) (the exterior carries u = 0)."""
    d = prob["dim"]
    hs = [(prob["hi"][a] - prob["lo"][a]) / (prob["n"][a] + 1) for a in range(d)]
    for a in range(1, d):
        if abs(hs[a] - hs[0]) > 1e-12 * hs[0]:
            raise ValueError("the 2D grid must have square cells")
    return hs[0]


def grid_points(prob: dict) -> np.ndarray:
    """Coordinates of the interior points in natural order (axis 0 fastest)."""
    d = prob["dim"]
    h = spacing(prob)
    axes = [prob["lo"][a] + h * np.arange(1, prob["n"][a] + 1) for a in range(d)]
    if d == 1:
        return axes[0][:, None]
    X0, X1 = np.meshgrid(axes[0], axes[1], indexing="xy")  # X0[i1, i0]
    return np.stack([X0.ravel(), X1.ravel()], axis=1)


def window_steps(prob: dict) -> int:
    """N_W with L_W = N_W h (reading of the symbol clash N / h = L_W / N)."""
    h = spacing(prob)
    q = prob["LW"] / h
    nw = int(round(q))
    if nw < 1 or abs(q - nw) > 1e-9 * max(1.0, q):
        raise ValueError("L_W must be a whole number of grid steps")
    return nw


def nu(prob: dict, r: np.ndarray) -> np.ndarray:
    """Levy density as a function of |y| (radial, symmetric kernels only).

    gauss : lam * exp(-eps^2 |y|^2)            (Merton jumps, Sec. H-matrix construction)
    stable: c_{d,s} / |y|^{d+2s}                (fractional Laplacian / alpha-stable)
    Zero beyond the truncation radius ``trunc`` (Eq. assumption)."""
    r = np.asarray(r, dtype=np.float64)
    d = prob["dim"]
    if prob["kernel"] == GAUSS:
        val = prob["lam"] * np.exp(-(prob["eps"] ** 2) * r * r)
    else:
        s = prob["s"]
        with np.errstate(divide="ignore"):
            val = c_ds(d, s) / r ** (d + 2.0 * s)
    trunc = _get(prob, "trunc", math.inf)
    return np.where(r <= trunc, val, 0.0)


def rho(r: np.ndarray, rr: float) -> np.ndarray:
    """Window function rho(y) = (1 - (|y|/r)^4)^3 for |y| < r, else 0.
    Meets Eq. rho_condition: 1 - rho = 3 (|y|/r)^4 + O(|y|^8) and rho = 0 for |y| >= r."""
    t = np.asarray(r, dtype=np.float64) / rr
    return np.where(t < 1.0, (1.0 - t ** 4) ** 3, 0.0)


def _window_offsets(prob: dict):
    """All nonzero window offsets j (integer, per axis) with their trapezoid
    weights w_j (h^d, halved on each window face coordinate; Eq. dl and the
    weights stated before Eq. I1approx)."""
    d = prob["dim"]
    h = spacing(prob)
    nw = window_steps(prob)
    j = np.arange(-nw, nw + 1)
    w1 = np.where(np.abs(j) == nw, 0.5, 1.0)
    if d == 1:
        J = j[:, None].astype(np.float64)
        W = w1 * h
    else:
        J0, J1 = np.meshgrid(j, j, indexing="ij")
        W0, W1 = np.meshgrid(w1, w1, indexing="ij")
        J = np.stack([J0.ravel(), J1.ravel()], axis=1).astype(np.float64)
        W = (W0 * W1).ravel() * h * h
    keep = np.any(J != 0, axis=1)
    return J[keep], W[keep]


def tail_mass(prob: dict) -> float:
    """T = integral of nu outside the window and inside the truncation radius
    (the u(x) part of I_2, Eq. I2approx).  1D: two half lines; 2D: polar
    integral over the square max-norm window, by adaptive quadrature."""
    d = prob["dim"]
    LW = prob["LW"]
    trunc = _get(prob, "trunc", math.inf)
    if d == 1:
        if trunc <= LW:
            return 0.0
        f = lambda y: float(nu(prob, np.array([y]))[0])
        val, _ = integrate.quad(f, LW, trunc, limit=400, epsabs=0.0, epsrel=1e-13)
        return 2.0 * val

    def radial(R):
        if R >= trunc:
            return 0.0
        if prob["kernel"] == STABLE:
            s = prob["s"]
            c = c_ds(2, s)
            hi = 0.0 if math.isinf(trunc) else trunc ** (-2.0 * s)
            return c * (R ** (-2.0 * s) - hi) / (2.0 * s)
        eps2 = prob["eps"] ** 2
        hi = 0.0 if math.isinf(trunc) else math.exp(-eps2 * trunc * trunc)
        return prob["lam"] * (math.exp(-eps2 * R * R) - hi) / (2.0 * eps2)

    # boundary of the square [-LW, LW]^2 at polar angle phi in [0, pi/4]
    g = lambda phi: radial(LW / math.cos(phi))
    val, _ = integrate.quad(g, 0.0, math.pi / 4.0, limit=400, epsabs=0.0, epsrel=1e-13)
    return 8.0 * val


def local_diffusion_integral(prob: dict) -> float:
    """Per-axis moment int rho(y) nu(y) y_d^2 dy of the subtracted term
    (Eq. evalIx1d / I3approx), by adaptive quadrature with the algebraic
    end-point weight of the singular kernel."""
    d = prob["dim"]
    s = prob["s"]
    rr = prob["r"]
    c = c_ds(d, s)
    # radial profile rho(t) t^{1-2s} on (0, r): the t^{1-2s} factor is the weight
    f = lambda t: (1.0 - (t / rr) ** 4) ** 3
    val, _ = integrate.quad(f, 0.0, rr, weight="alg", wvar=(1.0 - 2.0 * s, 0.0),
                            epsabs=0.0, epsrel=1e-13, limit=200)
    if d == 1:
        return 2.0 * c * val          # both half lines
    return 0.5 * 2.0 * math.pi * c * val  # half of the full |y|^2 moment per axis


def jump_constants(prob: dict):
    """Row-independent scalars of the discrete jump operator:
    lambda_W = sum' w_j nu(y_j) over the window (Eq. dl / first two sums of
    Eq. I1approx), T (Eq. I2approx) and kappa, the coefficient of the central
    second difference per axis from Eqs. I1approx and I3approx:
    kappa = (int rho nu y_d^2 - sum' w_j rho(y_j) nu(y_j) y_{j,d}^2) / (2 h^2).
    kappa = 0 for finite measures (no subtraction, Sec. Numerical Scheme)."""
    h = spacing(prob)
    J, W = _window_offsets(prob)
    Y = J * h
    R = np.sqrt(np.sum(Y * Y, axis=1))
    nuv = nu(prob, R)
    lam_w = float(np.sum(W * nuv))
    T = tail_mass(prob)
    kappa = 0.0
    if prob["kernel"] == STABLE:
        disc = float(np.sum(W * rho(R, prob["r"]) * nuv * Y[:, 0] ** 2))
        kappa = (local_diffusion_integral(prob) - disc) / (2.0 * h * h)
    return lam_w, T, kappa


def _grid_index(prob: dict) -> np.ndarray:
    """Integer grid coordinates of the interior points in natural order."""
    n = prob["n"]
    if prob["dim"] == 1:
        return np.arange(n[0])[:, None]
    i1, i0 = np.divmod(np.arange(n[0] * n[1]), n[0])
    return np.stack([i0, i1], axis=1)


def _row(prob: dict, consts, idx: np.ndarray, i: int) -> np.ndarray:
    d = prob["dim"]
    h = spacing(prob)
    nw = window_steps(prob)
    a = _get(prob, "a", 0.0)
    b = list(_get(prob, "b", [0.0, 0.0])) + [0.0, 0.0]
    cc = _get(prob, "c", 0.0)
    lam_w, T, kappa = consts
    J = idx - idx[i]                       # integer offsets to every grid point
    absJ = np.abs(J)
    w = np.full(idx.shape[0], h ** d)
    for ax in range(d):
        w = w * np.where(absJ[:, ax] == nw, 0.5, 1.0)
    R = np.sqrt(np.sum((J * h) ** 2, axis=1))
    row = w * nu(prob, R)
    for ax in range(d):
        for sgn in (+1, -1):
            k = np.nonzero((J[:, ax] == sgn) & (np.sum(absJ, axis=1) == 1))[0]
            if k.size:
                row[k[0]] += kappa + a / h ** 2 + sgn * b[ax] / (2.0 * h)
    row[i] = cc - 2.0 * d * a / h ** 2 - 2.0 * d * kappa - lam_w - T
    return row


def generator_dense(prob: dict) -> np.ndarray:
    """The dense N x N discrete generator G (natural order), row by row:

    G_ik = w(k-i) nu(|x_k - x_i|)                      k != i, k not an axis neighbour
    G_ik = the same + kappa + a/h^2 +- b_d/(2h)         k = i +- e_d
    G_ii = c - 2 d a / h^2 - 2 d kappa - lambda_W - T

    (Eq. Aij with the sign flipped, plus the singular corrections of
    Eqs. I1approx-I3approx).  Offsets beyond the window keep the plain weight
    h^d (they discretise the far field f_x^{L_W} of Eq. I2approx)."""
    consts = jump_constants(prob)
    idx = _grid_index(prob)
    N = idx.shape[0]
    G = np.empty((N, N))
    for i in range(N):
        G[i] = _row(prob, consts, idx, i)
    return G


def generator_dense_row(prob: dict, i: int) -> np.ndarray:
    """Row i of ``generator_dense`` without forming the whole matrix."""
    return _row(prob, jump_constants(prob), _grid_index(prob), i)


# ----------------------------------------------------------------------------
# Crank-Nicolson (Eq. scheme), dense direct method
# ----------------------------------------------------------------------------

def cn_solve(G: np.ndarray, u0: np.ndarray, dt: float, steps: int,
             forcing=None, step0: int = 0, literal: bool = True):
    """Advance u by ``steps`` CN steps: (I - theta G) u^{n+1} =
    (I + theta G) u^n + theta (f^n + f^{n+1}), theta = dt/2 (Eq. scheme; the
    trapezoidal forcing is this oracle's reading, the scheme has none).

    ``forcing(n)`` returns f at time level n (or None).  ``literal=False`` uses
    the identity (I + theta G) = 2 I - M, so only the LU of M is kept.
    Returns u at level step0 + steps."""
    theta = 0.5 * dt
    N = G.shape[0]
    M = np.eye(N) - theta * G
    lu = linalg.lu_factor(M, check_finite=False)
    P = None if not literal else np.eye(N) + theta * G
    u = np.array(u0, dtype=np.float64, copy=True)
    f_prev = forcing(step0) if forcing is not None else None
    for n in range(step0, step0 + steps):
        if forcing is not None:
            f_next = forcing(n + 1)
            extra = theta * (f_prev + f_next)
            f_prev = f_next
        else:
            extra = 0.0
        if literal:
            u = linalg.lu_solve(lu, P @ u + extra, check_finite=False)
        else:
            u = 2.0 * linalg.lu_solve(lu, u + 0.5 * extra, check_finite=False) - u
    return u


def cn_run_inplace(prob: dict, u0: np.ndarray, dt: float, steps: int, record=()):
    """The same Crank-Nicolson run as ``cn_solve(generator_dense(prob), u0, dt,
    steps, literal=False)`` (no forcing), holding a single N x N array: G is
    assembled, overwritten by M = I - theta G and factored in place (dense LU
    with partial pivoting), and each step takes u^{n+1} = 2 M^{-1} u^n - u^n,
    the identity form of Eq. scheme with (I + theta G) = 2 I - M.  For the
    largest grids the oracle reaches (N = 65536 needs one 34 GB array).
    Returns {level: u^level} for the levels in ``record`` and ``steps``."""
    theta = 0.5 * dt
    A = generator_dense(prob)
    A *= -theta
    A[np.diag_indices_from(A)] += 1.0
    # A is C-ordered, so A.T is the Fortran-ordered view LAPACK factors in
    # place: factor M^T and solve with trans=1, i.e. with M itself
    lu = linalg.lu_factor(A.T, overwrite_a=True, check_finite=False)
    u = np.array(u0, dtype=np.float64, copy=True)
    want = set(int(k) for k in record) | {int(steps)}
    out = {}
    if 0 in want:
        out[0] = u.copy()
    for n in range(steps):
        u = 2.0 * linalg.lu_solve(lu, u, trans=1, check_finite=False) - u
        if n + 1 in want:
            out[n + 1] = u.copy()
    return out
