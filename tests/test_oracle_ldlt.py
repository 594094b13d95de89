"""Pins for the oracle's complex-symmetric LDL^T without pivoting."""
import numpy as np
import pytest
import scipy.linalg as sl

import cc_problems as cp
from oracle import ldlt as D
from oracle import mesh as M
from oracle import system as S


def _system(p):
    m = M.lagrange_mesh(p.nlag, p.a)
    return S.assemble_dense(p, cp.potential_at(p, m["r"]), m)


def _unpivoted_lu(A):
    """Textbook right-looking elimination without row interchanges."""
    U = np.array(A, dtype=np.complex128, copy=True)
    n = U.shape[0]
    L = np.eye(n, dtype=np.complex128)
    for j in range(n):
        L[j + 1:, j] = U[j + 1:, j] / U[j, j]
        U[j + 1:, :] -= np.outer(L[j + 1:, j], U[j, :])
    return L, np.triu(U)


def test_ldlt_reconstructs_and_equals_unpivoted_lu():
    C, _ = _system(cp.config1())
    L, d = D.ldlt(C)
    assert np.allclose(np.tril(L), L) and np.all(np.diag(L) == 1)
    rec = (L * d[None, :]) @ L.T
    assert np.max(np.abs(rec - C)) < 1e-13 * np.max(np.abs(C))
    L2, U2 = _unpivoted_lu(C)
    assert np.max(np.abs(L2 - L)) < 1e-12
    assert np.max(np.abs(U2 - d[:, None] * L.T)) < 1e-12 * np.max(np.abs(C))


def test_ldlt_solve_matches_lapack():
    C, Phi = _system(cp.make_problem(12, 5, 30, 9.0))
    L, d = D.ldlt(C)
    X = D.ldlt_solve(L, d, Phi)
    Xr = sl.solve(C, Phi)
    assert np.max(np.abs(X - Xr)) / np.max(np.abs(Xr)) < 1e-9     # kappa ~1e6: both FP64


def test_hermitian_variant_is_caught():
    """Planted mistake: L D L^H (conjugated) does not reconstruct a complex-symmetric C."""
    C, _ = _system(cp.config1())
    L, d = D.ldlt(C)
    rec = (L * d[None, :]) @ L.conj().T
    assert np.max(np.abs(rec - C)) > 1e-6 * np.max(np.abs(C))


@pytest.mark.parametrize("W,bound", [(-10.0, 1.01), (-1.0, 1.01)])
def test_growth_on_the_config3_family(W, bound):
    """The kinetic diagonal dominates: no element growth without pivoting."""
    C, _ = _system(cp.config3(4, W=W))
    L, d = D.ldlt(C)
    assert D.growth(C, L, d) < bound
