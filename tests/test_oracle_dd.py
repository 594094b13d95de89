"""Pins for the double-double error-free transformations (exact rational checks)."""
from fractions import Fraction as Fr

import numpy as np

import cc_problems as cp
from oracle.ddarith import dd_div_d, dd_mul, dd_residual, two_prod, two_sum


def _vals(seed, n=400):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, n))
    edge = np.array([1.0, -1.0, 2.0**-52, 1 + 2.0**-52, 3.0, 1e300, -1e-300, 0.1, 1 / 3])
    return np.concatenate([v, edge])


def test_two_sum_two_prod_exact():
    a, b = _vals(1), _vals(2)[::-1].copy()
    s, e = two_sum(a, b)
    for i in range(a.size):
        assert Fr(s[i]) + Fr(e[i]) == Fr(a[i]) + Fr(b[i])
    # two_prod is exact while neither the product nor its error term underflows
    # and no factor exceeds 2^995 (Dekker's splitting)
    m = (np.abs(a) < 1e250) & (np.abs(b) < 1e250) & (np.abs(a * b) > 1e-250) & (np.abs(a * b) < 1e300)
    p, f = two_prod(a[m], b[m])
    for pa, pb, pp, pf in zip(a[m], b[m], p, f):
        assert Fr(pp) + Fr(pf) == Fr(pa) * Fr(pb)


def test_dd_mul_div_accuracy():
    a, b = _vals(3), _vals(4)
    m = (np.abs(a) < 1e100) & (np.abs(b) < 1e100) & (np.abs(b) > 1e-100) & (np.abs(a) > 1e-100)
    a, b = a[m], b[m]
    h, l = dd_mul(a, np.zeros_like(a), b, np.zeros_like(b))
    q, ql = dd_div_d(a, np.zeros_like(a), b)
    for i in range(a.size):
        ex = Fr(a[i]) * Fr(b[i])
        assert abs(Fr(h[i]) + Fr(l[i]) - ex) <= abs(ex) * Fr(2) ** -100
        exq = Fr(a[i]) / Fr(b[i])
        assert abs(Fr(q[i]) + Fr(ql[i]) - exq) <= abs(exq) * Fr(2) ** -100


def test_dd_residual_against_exact_rational():
    A, B = cp.random_dense(11, 6, nrhs=2)
    X = np.linalg.solve(A, B)
    r = dd_residual(A, X, B)
    for i in range(6):
        for j in range(2):
            er = Fr(B[i, j].real) - sum(Fr(A[i, k].real) * Fr(X[k, j].real) - Fr(A[i, k].imag) * Fr(X[k, j].imag) for k in range(6))
            ei = Fr(B[i, j].imag) - sum(Fr(A[i, k].real) * Fr(X[k, j].imag) + Fr(A[i, k].imag) * Fr(X[k, j].real) for k in range(6))
            # one final rounding of each part, plus the double-double accumulation
            # error ~2^-100 of the sum of the terms' magnitudes
            S = Fr(float(np.sum(np.abs(A[i]) * np.abs(X[:, j])) * 2 + abs(B[i, j])))
            assert abs(Fr(r[i, j].real) - er) <= abs(er) * Fr(2) ** -52 + S * Fr(2) ** -100
            assert abs(Fr(r[i, j].imag) - ei) <= abs(ei) * Fr(2) ** -52 + S * Fr(2) ** -100
