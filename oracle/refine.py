"""Reference ("truth") solution: FP64 LU plus double-double-residual refinement.

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

Iterative refinement as the paper describes it for its mixed-precision solver
(Sec. 3.2): solve with the stored factors, form r = b - M x in a higher
precision, solve M d = r with the same factors and update x <- x + d.  Here the
factors are complex128 (own LU of oracle.lu) and the residual is accumulated
in double-double (oracle.ddarith), so the refined x is accurate to about
u_64 * (1 + kappa * u_64) instead of kappa * u_64: the reference the GPU paths'
errors in X, R and U are measured against.

Pins (tests/test_oracle_refine.py): manufactured solutions x = 1 of
prescribed condition number (the paper's Fig. illcond construction) reach
|x - 1| ~ 1e-15 where plain LU leaves kappa * 1e-16.
"""
from __future__ import annotations

import numpy as np

from .ddarith import dd_residual
from .lu import lu_factor, lu_solve


def truth_solve(C: np.ndarray, B: np.ndarray, steps: int = 3):
    """Return (X, history) with history the max |r| / max |B| after each step."""
    LU, piv, info = lu_factor(C)
    if info:
        raise np.linalg.LinAlgError(f"exactly singular pivot at column {info}")
    X = lu_solve(LU, piv, B)
    scale = np.max(np.abs(B))
    hist = []
    for _ in range(steps):
        r = dd_residual(C, X, B)
        hist.append(float(np.max(np.abs(r)) / scale))
        X = X + lu_solve(LU, piv, r)
    hist.append(float(np.max(np.abs(dd_residual(C, X, B))) / scale))
    return X, hist


def truth_solve_structured(p, V, mesh=None, T0=None, steps: int = 2, residual=None):
    """Truth solution of C X = Phi for sizes where the oracle's own LU is out of reach.

    The factorisation is LAPACK's partial-pivoting zgetrf of the dense complex128 C
    (SciPy), the paper's own Type-1 solver (ZGESV, Sec. 3.1), used here as a library
    step; the refinement is the paper's (Sec. 3.2) with the residual formed through
    C's block structure in double-double (system.structured_residual_dd).
    ``residual(X) -> Phi - C X`` may replace that call (e.g. the same function
    evaluated on column chunks in parallel).  Returns (X, history, Phi) with history
    the max|r|/max|Phi| before each correction and after the last.

    Pins (tests/test_oracle_refine.py): equals truth_solve (own LU, dense
    double-double residual) on a system both can factor.
    """
    import scipy.linalg as sl

    from .mesh import kinetic_bloch, lagrange_mesh
    from .system import assemble_dense, structured_residual_dd

    m = mesh if mesh is not None else lagrange_mesh(p.nlag, p.a)
    T = T0 if T0 is not None else kinetic_bloch(p.nlag, p.a, m)
    C, Phi = assemble_dense(p, V, m, T)
    lu_piv = sl.lu_factor(C, overwrite_a=True, check_finite=False)
    del C
    if residual is None:
        def residual(X):
            return structured_residual_dd(p, V, X, Phi, m, T)
    X = sl.lu_solve(lu_piv, Phi, check_finite=False)
    scale = np.max(np.abs(Phi))
    hist = []
    for _ in range(steps):
        r = residual(X)
        hist.append(float(np.max(np.abs(r)) / scale))
        X = X + sl.lu_solve(lu_piv, r, check_finite=False)
    hist.append(float(np.max(np.abs(residual(X))) / scale))
    return X, hist, Phi
