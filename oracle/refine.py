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
