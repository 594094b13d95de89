"""GMRES-IR (RMAT_PARAM_REFINE = m > 0) on the GPU (-m gpu).

At kappa = 1e10 (the Householder-similarity construction of the paper's
conditioning study) the complex64 factors give cond * u_32 >> 1: classical
refinement stalls far above the FP64 level, while flexible GMRES
preconditioned by the same factors drives the FP64 residual to ~1e-15 and the
solution to the forward error kappa * u_64 of the exact x = 1.  On assembled
systems GMRES-IR must give the same X, R, U as the oracle's truth (every
precision, the Woodbury-kinetic method and charged channels included).
"""
import numpy as np
import pytest

import cc_problems as cp
from oracle import oracle_solve
from rmat_gpu import relerr, run_dense, run_problem

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10, 2: 1e-10, 3: 1e-10}


@pytest.fixture(scope="module")
def g():
    import paper_2512_11590_gb300 as mod
    mod.lib()
    return mod


@pytest.fixture()
def ctx(g):
    import torch
    torch.cuda.set_device(0)
    c = g.rmat_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    g.rmat_destroy(c)


@pytest.mark.parametrize("prec", [2, 3])
def test_gmres_ir_converges_where_classical_stalls(g, ctx, prec):
    A, B, Xe = cp.prescribed_kappa_hermitian(7, 512, 1e10, nrhs=3)
    g.rmat_set_param(ctx, g.RMAT_PARAM_REFINE, 0)
    classic = run_dense(ctx, A, B, prec, max_refine=20, tol=1e-14)
    g.rmat_set_param(ctx, g.RMAT_PARAM_REFINE, 30)
    gm = run_dense(ctx, A, B, prec, max_refine=20, tol=1e-14)
    inner = g.rmat_get_stats(ctx)["gmres_inner"]
    assert classic["rel"] > 1e-11                      # stalled (cond * u_32 ~ 600)
    assert gm["rel"] < 1e-13, (gm["rel"], gm["iters"], inner)
    assert relerr(gm["X"], Xe) < 1e-5                  # forward error ~ kappa * u_64
    assert inner > 0


CASES = {"config1": (cp.config1, 0), "nch16": (lambda: cp.config3(16), 0),
         "nch16-woodbury": (lambda: cp.config3(16), 1),
         "charged": (lambda: cp.charged_problem(34, 5, 80, 25.0), 0)}


@pytest.mark.parametrize("prec", [3, 1, 2, 0])
@pytest.mark.parametrize("case", list(CASES))
def test_gmres_ir_matches_oracle(g, ctx, case, prec):
    make, method = CASES[case]
    p = make()
    ref = oracle_solve(p, refine_steps=3)
    g.rmat_set_param(ctx, g.RMAT_PARAM_METHOD, method)
    g.rmat_set_param(ctx, g.RMAT_PARAM_REFINE, 20)
    out = run_problem(ctx, p, prec, max_refine=10, tol=1e-14)
    assert relerr(out["X"], ref["X"]) < TOL[prec]
    assert relerr(out["R"], ref["R"]) < TOL[prec]
    assert relerr(out["U"], ref["U"]) < TOL[prec]
    assert out["iters"] <= 4                           # outer corrections


def test_refine_param_range(g, ctx):
    for bad in (-1, 65):
        with pytest.raises(g.RmatError):
            g.rmat_set_param(ctx, g.RMAT_PARAM_REFINE, bad)


@pytest.mark.parametrize("case", ["config1", "nch16"])
def test_single_product_factor_under_gmres_ir(g, ctx, case):
    """RMAT_C64_1XF16_IR: the factor's trailing updates take one FP16 product (a third
    of the tensor work), so the factors are only ~u_16 cond(C) accurate; as the
    preconditioner of GMRES-IR they still give X, R, U at the refined bounds."""
    p = cp.config1() if case == "config1" else cp.config3(16)
    ref = oracle_solve(p, refine_steps=3)
    g.rmat_set_param(ctx, g.RMAT_PARAM_REFINE, 64)
    out = run_problem(ctx, p, g.RMAT_C64_1XF16_IR, max_refine=20, tol=1e-14)
    inner = g.rmat_get_stats(ctx)["gmres_inner"]
    print(f"1xF16 + GMRES-IR {case}: status {out['status']} outer {out['iters']} inner {inner:.0f}")
    assert out["status"] == g.RMAT_OK
    for k in ("X", "R", "U"):
        assert relerr(out[k], ref[k]) < 1e-10, k
