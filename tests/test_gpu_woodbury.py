"""Woodbury-kinetic method on the GPU (-m gpu): the factored matrix is
S = I + (K^-1 (x) I) W (Sec. 3.3, Type 3), the refinement keeps the FP64
residual of M, so X, R and U must match the oracle's truth to the same
tolerances as the direct method; the unrefined complex128 solve must equal the
oracle's own Schur-form solution (it is S, not M, that is factored); and the
refinement needs fewer corrections than the direct method (S is far better
conditioned than M)."""
import numpy as np
import pytest

import cc_problems as cp
from oracle import oracle_solve
from oracle import woodbury as WB
from rmat_gpu import relerr, run_problem

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
    g.rmat_set_param(c, g.RMAT_PARAM_METHOD, 1)
    yield c
    g.rmat_destroy(c)


def charged():
    p = cp.charged_problem(33, 6, 80, 30.0)
    p.thresh[-1] = 31.5                        # one closed channel
    return p


CASES = {"config1": cp.config1, "nch16": lambda: cp.config3(16),
         "ragged": lambda: cp.make_problem(61, 7, 37, 8.0), "charged": charged}


@pytest.mark.parametrize("prec", [0, 3, 1, 2])
@pytest.mark.parametrize("case", list(CASES))
def test_woodbury_matches_oracle(ctx, case, prec):
    p = CASES[case]()
    ref = oracle_solve(p, refine_steps=3)
    out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14)
    assert out["nopen"] == ref["nopen"]
    assert relerr(out["X"], ref["X"]) < TOL[prec]
    assert relerr(out["R"], ref["R"]) < TOL[prec]
    assert relerr(out["U"], ref["U"]) < TOL[prec]


def test_unrefined_c128_solve_is_the_schur_solution(ctx):
    p = cp.make_problem(62, 5, 40, 6.0)
    ref = oracle_solve(p, refine_steps=0)
    X_schur = WB.woodbury_solve(p, ref["V"], ref["mesh"], ref["T0"])
    out = run_problem(ctx, p, 0, max_refine=0, tol=0.0)
    assert relerr(out["X"], X_schur) < 1e-10


def test_fewer_corrections_than_direct(g, ctx):
    import torch
    p = cp.config3(16)
    wb = run_problem(ctx, p, 3, max_refine=30, tol=1e-13)
    c2 = g.rmat_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        direct = run_problem(c2, p, 3, max_refine=30, tol=1e-13)
    finally:
        g.rmat_destroy(c2)
    assert wb["iters"] < direct["iters"], (wb["iters"], direct["iters"])
    assert wb["iters"] <= 4


def test_method_and_mesh_switches_on_one_context(g, ctx):
    """Method 1 -> 0 -> 1 and a mesh change on one context: K^-1 is re-formed for
    the new mesh and nothing stale leaks between methods."""
    p1 = cp.config1()                          # nlag 50
    p2 = cp.make_problem(63, 3, 64, 9.0)       # nlag 64
    refs = {id(p): oracle_solve(p, refine_steps=3) for p in (p1, p2)}
    for method, p in [(1, p1), (0, p1), (1, p2), (1, p1)]:
        g.rmat_set_param(ctx, g.RMAT_PARAM_METHOD, method)
        out = run_problem(ctx, p, 3, max_refine=30, tol=1e-14)
        assert relerr(out["U"], refs[id(p)]["U"]) < 1e-10, (method, p.nlag)
