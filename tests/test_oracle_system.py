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


def _dd_case():
    from oracle.refine import truth_solve
    p = cp.make_problem(8, 6, 30, 12.0)
    m = M.lagrange_mesh(p.nlag, p.a)
    V = cp.potential_at(p, m["r"])
    C, Phi = S.assemble_dense(p, V, m)
    X, _ = truth_solve(C, Phi, steps=1)                  # residual ~1e-13: heavy cancellation
    return p, m, V, C, Phi, X


def test_channel_blocks_are_the_dense_blocks():
    p, m, V, C, Phi, X = _dd_case()
    Kb = S.channel_blocks(p, V, m)
    for al in range(p.nch):
        b = slice(al * p.nlag, (al + 1) * p.nlag)
        assert np.array_equal(C[b, b], Kb[al])


def test_structured_dd_residual_equals_dense_dd_residual():
    """Both sum the same exact products in double-double (~2^-104 of the terms), so
    they agree far below one ulp of the terms even where r cancels to 1e-13."""
    from oracle.ddarith import dd_residual
    p, m, V, C, Phi, X = _dd_case()
    r_dense = dd_residual(C, X, Phi)
    r_struct = S.structured_residual_dd(p, V, X, Phi, m)
    terms = np.max(np.abs(C) @ np.abs(X))
    assert np.max(np.abs(r_dense - r_struct)) <= 2.0 ** -100 * terms
    # the plain complex128 residual of the same X is wrong in its leading digits here
    assert np.max(np.abs(S.structured_residual(p, V, X, Phi, m) - r_dense)) > 1e3 * np.max(
        np.abs(r_dense - r_struct))


def test_structured_dd_residual_catches_a_dropped_term(monkeypatch):
    """Planted mistakes: one coupling channel or one kinetic column left out."""
    from oracle.ddarith import dd_residual
    p, m, V, C, Phi, X = _dd_case()
    r_dense = dd_residual(C, X, Phi)
    V2 = V.copy()
    V2[2, 4, :] = 0.0                                    # V_{4 2} dropped from the couplings
    r_bad = S.structured_residual_dd(p, V2, X, Phi, m)
    assert np.max(np.abs(r_bad - r_dense)) > 1e3 * np.max(np.abs(r_dense))
    Kb = S.channel_blocks(p, V, m)
    Kb[:, :, 7] = 0.0
    monkeypatch.setattr(S, "channel_blocks", lambda *a, **k: Kb)
    r_bad = S.structured_residual_dd(p, V, X, Phi, m)
    assert np.max(np.abs(r_bad - r_dense)) > 1e3 * np.max(np.abs(r_dense))
