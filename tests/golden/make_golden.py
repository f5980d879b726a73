"""Write the stored expected values under tests/golden/.

Calls only the oracle (the brute-force NUDFT, the exact definition the NUFFT
approximates, Section 2.1 Eq. 1) on seeded inputs from workloads.py.  Run from
the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def nudft_2d_tiny():
    Nd = (16, 8)
    om = W.uniform_random_om(40, 2, seed=11)
    x = W.complex_normal_image(Nd, seed=12)
    y = oracle.nudft_forward(om.astype(np.float64), x.astype(np.complex128))
    path = os.path.join(HERE, "nudft_2d_tiny.txt")
    with open(path, "w") as f:
        f.write("# Exact non-uniform DFT y_m = sum_n x[n] exp(-i sum_d om[m,d] (n_d - N_d/2))\n")
        f.write("# (the operator A approximates, Section 2.1 Eq. 1), written by make_golden.py\n")
        f.write("# inputs: Nd=16x8, om = workloads.uniform_random_om(40, 2, seed=11),\n")
        f.write("#         x = workloads.complex_normal_image((16, 8), seed=12)\n")
        f.write("# columns: m  re(y_m)  im(y_m)\n")
        for m, v in enumerate(y):
            f.write(f"{m} {v.real:.17e} {v.imag:.17e}\n")


if __name__ == "__main__":
    nudft_2d_tiny()
