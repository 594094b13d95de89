"""Pins for the oracle's truth refinement (double-double residual).

The manufactured right-hand side B = A 1 is itself rounded, so x = 1 is not
the exact solution of the stored system; the pin is a 50-digit mpmath solve of
the stored (A, B).
"""
import numpy as np
import pytest

import cc_problems as cp
from oracle.lu import solve
from oracle.refine import truth_solve


@pytest.mark.parametrize("kappa", [1e6, 1e10])
def test_refinement_reaches_double_precision(kappa):
    mp = pytest.importorskip("mpmath")
    n = 30
    A, B, _ = cp.prescribed_kappa_hermitian(9, n, kappa, nrhs=1)
    mp.mp.dps = 50
    Am = mp.matrix([[mp.mpc(complex(A[i, j])) for j in range(n)] for i in range(n)])
    Bm = mp.matrix([mp.mpc(complex(B[i, 0])) for i in range(n)])
    xm = mp.lu_solve(Am, Bm)
    xe = np.array([complex(xm[i]) for i in range(n)])
    X, hist = truth_solve(A, B, steps=3)
    e_ref = np.max(np.abs(X[:, 0] - xe)) / np.max(np.abs(xe))
    e_plain = np.max(np.abs(solve(A, B)[:, 0] - xe)) / np.max(np.abs(xe))
    assert e_ref < 3e-16                        # correctly rounded to within ~1 ulp
    assert e_plain > 10 * e_ref                 # plain LU is kappa-limited
    assert hist[-1] < 1e-15


def test_structured_truth_equals_dense_truth():
    """LAPACK factors + structured double-double residual reach the same solution as
    the oracle's own LU + dense double-double residual."""
    from oracle import mesh as M
    from oracle import system as S
    from oracle.refine import truth_solve_structured
    p = cp.make_problem(31, 8, 40, 9.0, W=-1.0)
    m = M.lagrange_mesh(p.nlag, p.a)
    V = cp.potential_at(p, m["r"])
    C, Phi = S.assemble_dense(p, V, m)
    X_ref, _ = truth_solve(C, Phi, steps=3)
    X, hist, Phi2 = truth_solve_structured(p, V, m, steps=2)
    assert np.array_equal(Phi, Phi2)
    assert np.max(np.abs(X - X_ref)) / np.max(np.abs(X_ref)) < 1e-15
    # r of the rounded solution is u |C||X|, not 0: the history only has to level off
    assert max(hist) < 1e-12
