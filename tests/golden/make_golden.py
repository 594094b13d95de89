"""Write tests/golden/config1_*.txt from the CPU oracle alone.

Config 1: nch=4, nlag=50 (N=200), a=15 fm, E=10 MeV, hm=20.9 MeV fm^2,
complex Woods-Saxon V0=-50, W=-10, R=4, ad=0.65, seeded couplings (seed 11590).
Values: the oracle's refined ("truth") R-matrix and collision matrix U,
real and imaginary parts, 17 significant digits.  Run from the repo root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import cc_problems as cp  # noqa: E402
from oracle import oracle_solve  # noqa: E402


def main():
    o = oracle_solve(cp.config1(), refine_steps=3)
    for name in ("R", "U"):
        M = o[name]
        np.savetxt(os.path.join(HERE, f"config1_{name}.txt"),
                   np.column_stack([M.real.ravel(), M.imag.ravel()]), fmt="%.17e",
                   header=f"config1 {name}: row-major {M.shape[0]}x{M.shape[1]}, columns re im; "
                          "written by tests/golden/make_golden.py from the CPU oracle")


if __name__ == "__main__":
    main()
