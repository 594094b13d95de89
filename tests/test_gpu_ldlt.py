"""Complex-symmetric LDL^T without pivoting on the tensor path (-m gpu).

C = C^T for every assembled problem (Sec. 2), so the factor C = L D L^T needs no
panel: each diagonal block is factored alone, the multipliers below it are
U12^T D11^-1, and the trailing updates keep only the tiles on or above the diagonal.
X is unique, so parity is judged on X, R and U against the oracle's pivoted solve,
for both tile widths of the symmetric update (128: one row tile per column tile on
the diagonal; 256: two), ragged tails and every tensor precision.
"""
import numpy as np
import pytest

import cc_problems as cp
from oracle import oracle_solve
from rmat_gpu import relerr, run_dense, run_problem

pytestmark = pytest.mark.gpu

TOL = {1: 1e-10, 3: 1e-10, 4: 1e-10}
_TRUTH = {}


@pytest.fixture(scope="module")
def g():
    import paper_2512_11590_gb300 as mod
    mod.lib()
    return mod


@pytest.fixture(scope="module")
def ctx(g):
    import torch
    torch.cuda.set_device(0)
    h = g.rmat_create(0, torch.cuda.current_stream().cuda_stream)
    yield h
    g.rmat_destroy(h)


def truth(p, key):
    if key not in _TRUTH:
        _TRUTH[key] = oracle_solve(p, refine_steps=3)
    return _TRUTH[key]


def with_params(g, ctx, params, fn):
    default = {g.RMAT_PARAM_PAIRED: 1}
    for k, v in params.items():
        g.rmat_set_param(ctx, k, v)
    try:
        return fn()
    finally:
        for k in params:
            g.rmat_set_param(ctx, k, default.get(k, 0))


@pytest.mark.parametrize("prec", [3, 1, 4])
@pytest.mark.parametrize("tc_bn", [256, 128])
@pytest.mark.parametrize("shape", [(16, 100), (29, 50), (3, 40)])
def test_ldlt_matches_oracle(g, ctx, prec, tc_bn, shape):
    """N = 1600 (12 full blocks and a 64-row tail), N = 1450 (11 and a 42-row tail),
    N = 120 (one block, no trailing update)."""
    nch, nlag = shape
    p = cp.make_problem(700 + nch, nch, nlag, 9.0)
    ref = truth(p, ("ldlt", nch, nlag))
    out = with_params(g, ctx, {g.RMAT_PARAM_FACTOR: 1, g.RMAT_PARAM_TC_BN: tc_bn},
                      lambda: run_problem(ctx, p, prec, max_refine=30, tol=1e-14, nb=128))
    st = g.rmat_get_stats(ctx)
    assert st["factor_ldlt"] == 1
    if p.N > 128:                           # multipliers below the first diagonal block
        assert 0 < st["ldlt_lmax"] < 4      # the kinetic diagonal dominates: small multipliers
    else:
        assert st["ldlt_lmax"] == 0
    assert out["info"] == 0
    assert out["status"] == g.RMAT_OK
    for k in ("X", "R", "U"):
        assert relerr(out[k], ref[k]) < TOL[prec], k


@pytest.mark.parametrize("paired", [1, 0])
@pytest.mark.parametrize("shape", [(16, 100), (29, 50), (5, 50)])
def test_ldlt_paired_and_single_updates(g, ctx, paired, shape):
    """Paired (two diagonal blocks per symmetric far update of depth 256, the default)
    and one update per block; N = 250 is a pair with a ragged second block."""
    nch, nlag = shape
    p = cp.make_problem(740 + nch, nch, nlag, 13.0)
    ref = truth(p, ("ldlt-pairs", nch, nlag))
    out = with_params(g, ctx, {g.RMAT_PARAM_FACTOR: 1, g.RMAT_PARAM_PAIRED: paired},
                      lambda: run_problem(ctx, p, 3, max_refine=30, tol=1e-14, nb=128))
    assert out["status"] == g.RMAT_OK
    for k in ("X", "R", "U"):
        assert relerr(out[k], ref[k]) < 1e-10, k


def test_ldlt_config3_block(g, ctx):
    """Config-3 family at N = 2400 (18 blocks and a 96-row tail): the same X, R and U
    as the pivoted factor."""
    p = cp.config3(nch=24, W=-10.0)
    ref = truth(p, ("ldlt-c3",))
    piv = run_problem(ctx, p, 3, max_refine=30, tol=1e-14, nb=128)
    assert g.rmat_get_stats(ctx)["factor_ldlt"] == 0
    out = with_params(g, ctx, {g.RMAT_PARAM_FACTOR: 1},
                      lambda: run_problem(ctx, p, 3, max_refine=30, tol=1e-14, nb=128))
    assert out["status"] == piv["status"] == g.RMAT_OK
    for k in ("X", "R", "U"):
        assert relerr(out[k], ref[k]) < 1e-10, k
        assert relerr(out[k], piv[k]) < 1e-10, k


def test_ldlt_loaded_symmetric_dense(g, ctx):
    """A loaded complex-symmetric matrix (not Hermitian) with a dominant diagonal."""
    rng = np.random.default_rng(77)
    n, nrhs = 700, 6
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = (M + M.T) / 2 + np.diag(40.0 + 10j * rng.standard_normal(n))
    B = rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))
    X0 = np.linalg.solve(A, B)
    out = with_params(g, ctx, {g.RMAT_PARAM_FACTOR: 1},
                      lambda: run_dense(ctx, A, B, 3, max_refine=30, tol=1e-14, nb=128))
    assert out["status"] == g.RMAT_OK
    assert relerr(out["X"], X0) < 1e-11


def test_factor_param_rejects_bad_value(g, ctx):
    import ctypes as ct
    assert g.lib().rmat_set_param(ct.c_void_p(ctx), g.RMAT_PARAM_FACTOR, 2) == -3
