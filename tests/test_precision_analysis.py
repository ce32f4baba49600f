"""The precision question of the Crank-Nicolson path, answered on the dense
oracle (CPU): where single precision can and cannot stand in for FP64 on the
1D Levy workload (drift 0.3, sigma 0.2, alpha = 1.5 truncated to |y| <= 2),
here at N = 2047, dt = 1e-3, 200 steps from u0 = exp(-50 x^2).

* The right-hand side u + dt/2 G u cannot use FP32 entries: G's diffusion
  rows hold a/h^2 ~ 2e7 and sum to O(1), so even with FP64 accumulation the
  rounding of the stored entries leaves ~1e-4 after 200 steps, and no
  refinement of the solve recovers it (the right-hand side itself is wrong).
* The factors can be FP32 if each solve is refined against the FP64
  operator: one sweep brings the error to ~1e-9, two to round-off.

So a mixed path costs at least one extra FP64 matvec and solve per step,
while the solve it would cheapen is latency-bound, not bandwidth-bound."""
import numpy as np
import pytest
from scipy import linalg

from oracle import levy_dense as O
from paper_1812_08324_gb300 import workloads as W

N, DT, STEPS = 2047, 1e-3, 200


@pytest.fixture(scope="module")
def setup():
    prob = W.levy_1d(N)
    G = O.generator_dense(prob)
    th = 0.5 * DT
    M = np.eye(N) - th * G
    lu = linalg.lu_factor(M)
    u0 = W.gaussian_u0(prob, 50.0)

    def run(matvec, solve):
        u = u0.copy()
        for _ in range(STEPS):
            u = solve(u + th * matvec(u))
        return u

    ref = run(lambda u: G @ u, lambda r: linalg.lu_solve(lu, r))
    return G, M, lu, run, ref


def _err(u, ref):
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


def test_fp32_entries_in_the_rhs_matvec_fail(setup):
    G, M, lu, run, ref = setup
    G32 = G.astype(np.float32).astype(np.float64)      # FP32 storage, FP64 accumulation
    u = run(lambda v: G32 @ v, lambda r: linalg.lu_solve(lu, r))
    assert _err(u, ref) > 1e-5


def test_fp32_factors_need_refinement(setup):
    G, M, lu, run, ref = setup
    lu32 = linalg.lu_factor(M.astype(np.float32))

    def solve(r, sweeps):
        z = linalg.lu_solve(lu32, r.astype(np.float32)).astype(np.float64)
        for _ in range(sweeps):
            z = z + linalg.lu_solve(lu32, (r - M @ z).astype(np.float32)).astype(np.float64)
        return z

    errs = [_err(run(lambda v: G @ v, lambda r, s=s: solve(r, s)), ref) for s in (0, 1, 2)]
    assert errs[0] > 1e-5           # FP32 factors alone miss the 1e-6 target
    assert errs[1] < 1e-8           # one FP64 refinement sweep per step recovers it
    assert errs[2] < 1e-11          # two reach round-off
