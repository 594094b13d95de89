"""Partial-pivoting LU factorisation and triangular solves (oracle).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

The paper's Type-1 solver factors M = P L U with partial pivoting, L unit
lower triangular and U upper triangular, then solves for all nch right-hand
sides by forward and backward substitution (Sec. 3.1, Eq. for M = P L U).
The paper does not state the pivot measure; this oracle uses |Re| + |Im|
(LAPACK's izamax measure for ZGETRF) and takes the FIRST row attaining the
maximum on ties.  Elimination is the textbook unblocked right-looking order:
for each column j pick the pivot, swap whole rows, divide the column below
the diagonal by the pivot and subtract the rank-1 update.

Pins (tests/test_oracle_lu.py): brute-force inverse on tiny systems,
LAPACK zgesv / zgetrf via SciPy (pivot vector and solution), P L U = A
reconstruction, and manufactured x = 1 solutions of prescribed condition.
"""
from __future__ import annotations

import numpy as np


def cabs1(z):
    return np.abs(z.real) + np.abs(z.imag)


def lu_factor(A: np.ndarray):
    """Return (LU, piv, info).

    LU holds L (strictly lower, unit diagonal implied) and U; piv[j] is the
    0-based row swapped with row j at step j (LAPACK ipiv, 0-based).  info is
    0, or k > 0 (1-based) for the first exactly zero pivot, in which case the
    column is left unscaled and elimination continues (LAPACK convention).
    """
    LU = np.array(A, dtype=np.complex128, copy=True)
    n = LU.shape[0]
    piv = np.zeros(n, dtype=np.int64)
    info = 0
    for j in range(n):
        p = j + int(np.argmax(cabs1(LU[j:, j])))      # argmax returns the first maximum
        piv[j] = p
        if p != j:
            LU[[j, p], :] = LU[[p, j], :]
        pivot = LU[j, j]
        if pivot == 0:
            if info == 0:
                info = j + 1
            continue
        LU[j + 1:, j] = LU[j + 1:, j] / pivot
        LU[j + 1:, j + 1:] -= np.outer(LU[j + 1:, j], LU[j, j + 1:])
    return LU, piv, info


def apply_pivots(piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    """P^T B: apply the row interchanges in order j = 0..n-1."""
    Y = np.array(B, dtype=np.complex128, copy=True)
    for j, p in enumerate(piv):
        if p != j:
            Y[[j, p], :] = Y[[p, j], :]
    return Y


def lu_solve(LU: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve A X = B with the factors of ``lu_factor`` (forward then backward)."""
    n = LU.shape[0]
    Y = apply_pivots(piv, B)
    if Y.ndim == 1:
        Y = Y[:, None]
    for i in range(1, n):                              # L y = P^T b, unit diagonal
        Y[i, :] -= LU[i, :i] @ Y[:i, :]
    for i in range(n - 1, -1, -1):                     # U x = y
        Y[i, :] = (Y[i, :] - LU[i, i + 1:] @ Y[i + 1:, :]) / LU[i, i]
    return Y if B.ndim == 2 else Y[:, 0]


def solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    LU, piv, info = lu_factor(A)
    if info:
        raise np.linalg.LinAlgError(f"exactly singular pivot at column {info}")
    return lu_solve(LU, piv, B)
