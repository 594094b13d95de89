"""Complex-symmetric LDL^T factorisation without pivoting (oracle).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

The internal-region matrix of Eq. (block_structure) is complex symmetric, C = C^T
(not Hermitian: the transpose, no conjugation), so it has the factorisation
C = L D L^T with L unit lower triangular and D diagonal whenever no leading
principal minor vanishes.  Written out column by column (j = 0, 1, ...):

  d_j      = C[j, j] - sum_{k<j} L[j, k]^2 d_k
  L[i, j]  = (C[i, j] - sum_{k<j} L[i, k] L[j, k] d_k) / d_j,   i > j.

Without pivoting this is the unpivoted LU with U = D L^T; it is stable when the
diagonal dominates, as the kinetic diagonal does on this family (growth factor
1.0 on config 3; not on config 3b, where refinement with the complex64 factor
contracts only ~3x per step).  The paper's solvers pivot (Sec. 3.1); this is the
symmetric variant of the next-step list, for systems whose diagonal dominates.

Pins (tests/test_oracle_ldlt.py): L D L^T reconstructs C; U = D L^T equals the
unpivoted LU of the oracle's own elimination; the solve matches LAPACK; a
conjugated transpose (the Hermitian factorisation) fails the reconstruction.
"""
from __future__ import annotations

import numpy as np


def ldlt(C: np.ndarray):
    """Return (L, d): L unit lower triangular, d the diagonal of D, C = L diag(d) L^T."""
    C = np.asarray(C, dtype=np.complex128)
    n = C.shape[0]
    L = np.eye(n, dtype=np.complex128)
    d = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        d[j] = C[j, j] - np.sum(L[j, :j] ** 2 * d[:j])
        if d[j] == 0:
            raise np.linalg.LinAlgError(f"zero pivot at column {j + 1}")
        L[j + 1:, j] = (C[j + 1:, j] - (L[j + 1:, :j] * d[:j]) @ L[j, :j]) / d[j]
    return L, d


def ldlt_solve(L: np.ndarray, d: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = (L D L^T)^-1 B by forward substitution, diagonal scaling, backward substitution."""
    n = L.shape[0]
    Y = np.array(B, dtype=np.complex128, copy=True)
    for i in range(n):
        Y[i] -= L[i, :i] @ Y[:i]
    Y /= d[:, None] if Y.ndim == 2 else d
    for i in range(n - 1, -1, -1):
        Y[i] -= L[i + 1:, i] @ Y[i + 1:]
    return Y


def growth(C: np.ndarray, L: np.ndarray, d: np.ndarray) -> float:
    """max |U| / max |C| with U = D L^T (the element growth of the elimination)."""
    U = d[:, None] * L.T
    return float(np.max(np.abs(U)) / np.max(np.abs(C)))
