"""Writes the dense-oracle solutions of the 1D Levy workload (drift 0.3,
diffusion sigma = 0.2, alpha-stable jumps alpha = 1.5 truncated to |y| <= 2,
u0 = exp(-50 x^2), dt = 1e-3) that the GPU parity tests and the benchmark's
accuracy figure compare against.  Calls only the oracle (inputs from the
workload descriptions).  Each output file ``levy1d_n{N}_dt1e-3.npz`` holds
arrays ``u{k}`` = u at level k in natural grid order.

    python tests/golden/make_levy1d_golden.py 32768 20,1000

N = 32768 holds one 8.6 GB array and runs for about 20 minutes on 8 cores.
The workload's own N = 65536 (a 34 GB array) is out of reach: the host
LAPACK's LU fails on matrices of more than 2^32 entries.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import levy_dense as O  # noqa: E402
from paper_1812_08324_gb300 import workloads as W  # noqa: E402


def main():
    n = int(sys.argv[1])
    levels = [int(x) for x in sys.argv[2].split(",")]
    prob = W.levy_1d(n)
    u0 = W.gaussian_u0(prob, 50.0)
    t0 = time.time()
    res = O.cn_run_inplace(prob, u0, 1e-3, max(levels), record=levels)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"levy1d_n{n}_dt1e-3.npz")
    np.savez_compressed(out, **{f"u{k}": res[k] for k in levels})
    print(f"wrote {out} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
