"""Writes the dense-oracle solution of the 2D fractional Laplacian workload
(order s, homogeneous Dirichlet exterior on the unit square, grid side n,
u0 = the Gaussian bump of sigma 0.1, dt = 1/200) that the 2D GPU parity test
and the benchmark's 2D accuracy figure compare against.  Calls only the oracle
(inputs from the workload descriptions).  The output file
``frac2d_n{n}_s{s}_dt5e-3.npz`` holds arrays ``u{k}`` = u at level k in
natural grid order.

    python tests/golden/make_frac2d_golden.py 128 0.75 20,200

Side 128 (N = 16384) holds one 2.1 GB array and runs for a few minutes on
8 cores; the workload's own side 256 (N = 65536) needs 34 GB and more than
2^32 entries, which the host LAPACK's LU does not take.
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
    s = float(sys.argv[2])
    levels = [int(x) for x in sys.argv[3].split(",")]
    prob = W.frac_lap_2d(n, s)
    u0 = W.initial_data(prob, "bump")
    t0 = time.time()
    res = O.cn_run_inplace(prob, u0, 1.0 / 200, max(levels), record=levels)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"frac2d_n{n}_s{s}_dt5e-3.npz")
    np.savez_compressed(out, **{f"u{k}": res[k] for k in levels})
    print(f"wrote {out} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
