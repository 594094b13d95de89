"""Pins for the oracle's matrix assembly and structured residual (Eq. block_structure)."""
import numpy as np

import cc_problems as cp
from oracle import mesh as M
from oracle import system as S


def test_structure_and_symmetry():
    p = cp.config1()
    m = M.lagrange_mesh(p.nlag, p.a)
    V = cp.potential_at(p, m["r"])
    C, Phi = S.assemble_dense(p, V, m)
    assert np.array_equal(C, C.T)                       # complex symmetric, exactly
    n = p.nlag
    # off-diagonal channel blocks are diagonal (local coupling, Lagrange property)
    blk = C[0:n, n:2 * n]
    assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0
    # fraction of nonzeros ~ (nch*nlag^2 + nch(nch-1) nlag) / N^2
    nnz = np.count_nonzero(C)
    assert nnz <= p.nch * n * n + p.nch * (p.nch - 1) * n
    assert np.array_equal(Phi[:n, 0], m["f_a"]) and np.count_nonzero(Phi[n:, 0]) == 0


def test_structured_residual_equals_dense():
    p = cp.make_problem(8, 6, 30, 12.0)
    m = M.lagrange_mesh(p.nlag, p.a)
    V = cp.potential_at(p, m["r"])
    C, Phi = S.assemble_dense(p, V, m)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((p.N, p.nch)) + 1j * rng.standard_normal((p.N, p.nch))
    r_dense = S.dense_residual(C, X, Phi)
    r_struct = S.structured_residual(p, V, X, Phi, m)
    assert np.max(np.abs(r_dense - r_struct)) < 1e-14 * np.max(np.abs(C)) * np.max(np.abs(X))
