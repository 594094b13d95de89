"""The oracle reproduces its committed config-1 golden values (regression pin)."""
import os

import numpy as np

import cc_problems as cp
from oracle import oracle_solve

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    a = np.loadtxt(os.path.join(GOLD, f"config1_{name}.txt"))
    z = a[:, 0] + 1j * a[:, 1]
    n = int(round(np.sqrt(z.size)))
    return z.reshape(n, n)


def test_config1_golden():
    o = oracle_solve(cp.config1(), refine_steps=3)
    for name in ("R", "U"):
        g = load(name)
        assert np.max(np.abs(o[name] - g)) <= 1e-14 * np.max(np.abs(g))
