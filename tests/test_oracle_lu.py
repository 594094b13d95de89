"""Pins for the oracle's partial-pivoting LU and solves (Sec. 3.1, M = P L U).

Independent references: brute-force inversion, LAPACK zgetrf/zgesv through
SciPy, exact reconstruction P L U = A, and manufactured solutions.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import cc_problems as cp
from oracle.lu import apply_pivots, lu_factor, lu_solve, solve


def _PLU(LU, piv):
    n = LU.shape[0]
    Lm = np.tril(LU, -1) + np.eye(n)
    Um = np.triu(LU)
    return apply_pivots(piv, np.eye(n)).T @ (Lm @ Um)     # P = (P^T)^T


@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_brute_force_inverse(n):
    A, B = cp.random_dense(7 + n, n, nrhs=3)
    X = solve(A, B)
    Xb = np.linalg.inv(A) @ B
    assert np.max(np.abs(X - Xb)) < 1e-12 * np.max(np.abs(Xb))


@pytest.mark.parametrize("n", [8, 40, 97])
def test_matches_lapack_pivots_and_solution(n):
    A, B = cp.random_dense(100 + n, n, nrhs=5)
    LU, piv, info = lu_factor(A)
    lu_l, piv_l = sla.lu_factor(A)            # LAPACK zgetrf: |Re|+|Im| pivots
    assert info == 0
    assert np.array_equal(piv, piv_l)
    assert np.max(np.abs(LU - lu_l)) < 1e-11 * np.max(np.abs(lu_l))
    X = lu_solve(LU, piv, B)
    Xl = sla.solve(A, B)
    assert np.max(np.abs(X - Xl)) < 1e-11 * np.max(np.abs(Xl))


def test_reconstruction_PLU():
    A, _ = cp.random_dense(3, 30)
    LU, piv, _ = lu_factor(A)
    assert np.max(np.abs(_PLU(LU, piv) - A)) < 1e-13 * np.max(np.abs(A))


def test_pivot_measure_is_cabs1_first_index_on_ties():
    # column 0: |1+3i| has the largest modulus but |Re|+|Im| ties 4 = 4 = 4
    A = np.array([[1.0 + 0j, 0, 0],
                  [2.0 + 2.0j, 1, 0],
                  [1.0 + 3.0j, 0, 1],
                  ], dtype=np.complex128)
    A = np.vstack([A, [[4.0 + 0j, 0, 2]]])[:3]          # keep 3x3
    A[0, 0] = 4.0
    _, piv, _ = lu_factor(A)
    assert piv[0] == 0                                   # first of the three cabs1 = 4 rows
    B = np.array([[0.5, 0, 0], [3.0 + 1j, 1, 0], [1.0 + 3j, 0, 1]], dtype=np.complex128)
    _, piv, _ = lu_factor(B)
    assert piv[0] == 1                                   # cabs1 4 beats |1+3i| (cabs1 4): first wins


def test_zero_pivot_reports_info():
    A = np.array([[0, 0], [0, 1]], dtype=np.complex128)
    _, _, info = lu_factor(A)
    assert info == 1


@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10])
def test_manufactured_prescribed_condition(kappa):
    A, B, Xe = cp.prescribed_kappa_hermitian(5, 60, kappa, nrhs=2)
    assert abs(np.linalg.cond(A) / kappa - 1) < 1e-3
    X = solve(A, B)
    assert np.max(np.abs(X - Xe)) < 50 * kappa * 1.1e-16
