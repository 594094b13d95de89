"""GPU parity against the CPU oracle, through the C ABI (-m gpu).

Tolerances (max|dU| / max|U_truth|, truth = oracle FP64 LU + double-double
refinement): 1e-12 for the complex128 path after FP64 refinement, 1e-10 for
the complex64 paths after FP64 refinement (the paper's FP64-vs-mixed targets).
The solution X and the R-matrix are held to the same bounds.
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


@pytest.fixture(scope="module")
def ctx(g):
    import torch
    torch.cuda.set_device(0)
    h = g.rmat_create(0, torch.cuda.current_stream().cuda_stream)
    yield h
    g.rmat_destroy(h)


_TRUTH = {}


def truth(p, key):
    if key not in _TRUTH:
        _TRUTH[key] = oracle_solve(p, refine_steps=3)
    return _TRUTH[key]


PRECS = [0, 1, 2, 3]


@pytest.mark.parametrize("prec", PRECS)
def test_config1_vs_oracle(g, ctx, prec):
    p = cp.config1()
    ref = truth(p, "c1")
    out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14)
    assert out["info"] == 0
    assert out["nopen"] == ref["nopen"] == 4
    for k in ("U", "R", "X"):
        e = relerr(out[k], ref[k])
        assert e < TOL[prec], (k, e)
    lu_only = run_problem(ctx, p, prec, max_refine=0)
    e0 = relerr(lu_only["U"], ref["U"])
    assert e0 < (1e-9 if prec == 0 else 1e-2)     # LU alone: FP64 ~ kappa u_64, FP32 ~ kappa u_32


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nch,nlag,nb", [(5, 37, 32), (3, 50, 64), (7, 23, 32), (1, 40, 32)])
def test_ragged_multi_panel(g, ctx, prec, nch, nlag, nb):
    p = cp.make_problem(1000 + nch * nlag, nch, nlag, 12.0)
    ref = truth(p, ("rag", nch, nlag))
    out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14, nb=nb)
    for k in ("U", "R"):
        assert relerr(out[k], ref[k]) < TOL[prec], k


@pytest.mark.parametrize("prec", PRECS)
def test_closed_channels(g, ctx, prec):
    p = cp.config1()
    p.E = 3.0
    p.thresh = np.array([0.0, 1.0, 4.0, 4.5])
    ref = truth(p, "closed")
    out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14)
    assert out["nopen"] == 2
    assert relerr(out["U"], ref["U"]) < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_nch16_nlag100_many_tiles(g, ctx, prec):
    p = cp.config2(16)                      # N = 1600, 16 right-hand sides
    ref = truth(p, "c2-16")
    out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14)
    for k in ("U", "R"):
        assert relerr(out[k], ref[k]) < TOL[prec], k


@pytest.mark.parametrize("prec", PRECS)
def test_dense_pivoting_vs_lapack(g, ctx, prec):
    A, B = cp.random_dense(77, 300, nrhs=3)
    Xe = np.linalg.solve(A, B)
    out = run_dense(ctx, A, B, prec, max_refine=20, tol=1e-15, nb=64)
    assert relerr(out["X"], Xe) < 1e-12


def test_prescribed_condition_refinement(g, ctx):
    """kappa = 1e6 Hermitian system (the paper's Fig. illcond construction):
    the FP32 factor alone is kappa*u_32-limited; FP64-residual refinement brings
    the solution to the FP64 level kappa*u_64 of the double-double truth."""
    from oracle.refine import truth_solve
    A, B, _ = cp.prescribed_kappa_hermitian(3, 256, 1e6, nrhs=2)
    Xe, _ = truth_solve(A, B, steps=2)
    plain = run_dense(ctx, A, B, 2, max_refine=0)
    ref = run_dense(ctx, A, B, 2, max_refine=30, tol=1e-15)
    assert ref["iters"] >= 1
    assert relerr(ref["X"], Xe) < 1e-9
    assert relerr(plain["X"], Xe) > 1e-7


def test_exactly_singular_reports_info(g, ctx):
    A, B = cp.random_dense(5, 64, nrhs=1)
    A[:, 10] = 0.0
    out = run_dense(ctx, A, B, 0, nb=32)
    assert out["factor_status"] == g.RMAT_ESINGULAR and out["info"] == 11


def test_bounded_panel_wait_times_out_cleanly(g, ctx):
    """A panel barrier with a 1-poll limit gives up and reports RMAT_ETIMEOUT;
    the context stays usable afterwards (no hang, no fault)."""
    import torch
    A, B = cp.random_dense(9, 2048, nrhs=1)
    g.rmat_set_param(ctx, g.RMAT_PARAM_PANEL_CTAS, 8)
    g.rmat_set_param(ctx, g.RMAT_PARAM_SPIN_LIMIT, 1)
    try:
        Ad = torch.from_numpy(np.asfortranarray(A).ravel(order="F")).cuda()
        Bd = torch.from_numpy(np.asfortranarray(B).ravel(order="F")).cuda()
        g.rmat_load_dense(ctx, 2048, 1, Ad.data_ptr(), 2048, Bd.data_ptr(), 2048, 0)
        import ctypes as ct
        info = ct.c_int(0)
        s = g.lib().rmat_factor(ct.c_void_p(ctx), ct.byref(info))
        assert s == g.RMAT_ETIMEOUT
    finally:
        g.rmat_set_param(ctx, g.RMAT_PARAM_SPIN_LIMIT, 20000000)
        g.rmat_set_param(ctx, g.RMAT_PARAM_PANEL_CTAS, 0)
    out = run_dense(ctx, A[:200, :200], B[:200], 0)
    assert relerr(out["X"], np.linalg.solve(A[:200, :200], B[:200])) < 1e-12


@pytest.mark.parametrize("prec,nb", [(1, 32), (1, 128), (2, 128), (0, 32), (0, 64), (3, 64),
                                     (3, 128)])
def test_block_widths(g, ctx, prec, nb):
    p = cp.config2(16)
    ref = truth(p, "c2-16")
    out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14, nb=nb)
    assert relerr(out["U"], ref["U"]) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("equil", [0, 1])
def test_equilibration_switch(g, ctx, equil, prec):
    p = cp.config3(16, W=-1.0)               # config 3b: weaker absorption, worse conditioned
    ref = truth(p, "c3b-16")
    g.rmat_set_param(ctx, g.RMAT_PARAM_EQUILIBRATE, equil)
    try:
        out = run_problem(ctx, p, prec, max_refine=40, tol=1e-14)
        hist = g.rmat_refine_history(ctx)
        berr = g.rmat_get_stats(ctx)["backward_error"]
    finally:
        g.rmat_set_param(ctx, g.RMAT_PARAM_EQUILIBRATE, -1)
    assert relerr(out["U"], ref["U"]) < TOL[prec]
    # stopped at the FP64 floor: one correction after the floor-level residual
    assert out["status"] == g.RMAT_OK and berr <= 0.5 * 2.0 ** -53
    assert len(hist) == out["iters"]


@pytest.mark.parametrize("scale_a,scale_b", [(1e7, 1e-12), (1e-6, 1e9)])
def test_fp16_planes_far_outside_fp16_range(g, ctx, scale_a, scale_b):
    """Split-FP16 tensor path on a dense system whose entries (scale_a) and right-hand
    sides (scale_b) lie far outside the FP16 range: the per-block and per-column
    power-of-two scales keep every operand representable, and refinement reaches
    the FP64 level (checked against LAPACK)."""
    A, B = cp.random_dense(31, 640, nrhs=4)
    A, B = A * scale_a, B * scale_b
    Xe = np.linalg.solve(A, B)
    out = run_dense(ctx, A, B, 3, max_refine=30, tol=1e-15, nb=128)
    assert out["iters"] >= 1
    assert relerr(out["X"], Xe) < 1e-12


@pytest.mark.parametrize("prec", [3, 0])
def test_grid_panel_variant(g, ctx, prec):
    """A fixed panel CTA count selects the cooperative grid-barrier panel (used for
    panels taller than one cluster's shared memory); same results as the default."""
    p = cp.config2(16)
    ref = truth(p, "c2-16")
    g.rmat_set_param(ctx, g.RMAT_PARAM_PANEL_CTAS, 16)
    try:
        out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14)
    finally:
        g.rmat_set_param(ctx, g.RMAT_PARAM_PANEL_CTAS, 0)
    assert relerr(out["U"], ref["U"]) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("paired,nb", [(0, 64), (1, 64), (1, 128)])
def test_paired_trailing_updates(g, ctx, prec, paired, nb):
    """Two panels per tensor-core trailing update (K = 2 nb, interchanges of the
    second panel applied to a copy of the first panel's L21) and one update per
    panel both reach the oracle's U."""
    p = cp.config2(16)
    ref = truth(p, "c2-16")
    g.rmat_set_param(ctx, g.RMAT_PARAM_PAIRED, paired)
    try:
        out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14, nb=nb)
    finally:
        g.rmat_set_param(ctx, g.RMAT_PARAM_PAIRED, 1)
    assert relerr(out["U"], ref["U"]) < TOL[prec]
    assert relerr(out["X"], ref["X"]) < TOL[prec]


@pytest.mark.parametrize("prec,nb,ctas", [(3, 128, 2), (3, 64, 3), (1, 128, 2), (0, 64, 2)])
def test_panel_rows_in_global_memory(g, ctx, prec, nb, ctas):
    """Few panel CTAs, so each holds too many rows for shared memory: the grid panel
    works on its rows in global memory (the variant the first panels of N = 51200 use)."""
    p = cp.config2(16)
    ref = truth(p, "c2-16")
    g.rmat_set_param(ctx, g.RMAT_PARAM_PANEL_CTAS, ctas)
    try:
        out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14, nb=nb)
    finally:
        g.rmat_set_param(ctx, g.RMAT_PARAM_PANEL_CTAS, 0)
    assert relerr(out["U"], ref["U"]) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("nb,shape", [(64, (16, 100)), (128, (16, 100)), (128, (29, 50))])
def test_solve_lookahead_vs_oracle(g, prec, mode, nb, shape):
    """RMAT_PARAM_SOLVE_LOOKAHEAD = 1: next-step updates on the main stream (K split
    over CTAs), = 2: inside the diagonal-block application (atomic, CUDA cores); far
    rows on the side stream, double-buffered Y planes; with block width 128 the steps
    are pairs of blocks (N = 1450: five pairs, one single block and a 42-row tail);
    same tolerances."""
    import torch
    torch.cuda.set_device(0)
    nch, nlag = shape
    p = cp.config3(16) if shape == (16, 100) else cp.make_problem(900 + nch, nch, nlag, 11.0)
    ref = truth(p, "c3-16" if shape == (16, 100) else ("steps", nch, nlag))
    h = g.rmat_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        g.rmat_set_param(h, g.RMAT_PARAM_SOLVE_LOOKAHEAD, mode)
        out = run_problem(h, p, prec, max_refine=30, tol=1e-14, nb=nb)
    finally:
        g.rmat_destroy(h)
    assert out["status"] == g.RMAT_OK
    for k in ("U", "R", "X"):
        e = relerr(out[k], ref[k])
        assert e < TOL[prec], (k, e)


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("groups", [1, 2])
@pytest.mark.parametrize("nb", [64, 128])
def test_solve_column_groups_vs_oracle(g, prec, groups, nb):
    """RMAT_PARAM_SOLVE_GROUPS = 2: the 256 right-hand sides of nch = 256 channels in two
    column groups of 128, each with its own sweeps, Y-plane rows, column scales and
    stream pair, running concurrently (N = 1536: 12 blocks of 128 or 24 of 64, look-ahead
    on); same tolerances as one group."""
    import torch
    torch.cuda.set_device(0)
    p = cp.make_problem(977, 256, 6, 10.0)
    ref = truth(p, ("groups", 256, 6))
    h = g.rmat_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        g.rmat_set_param(h, g.RMAT_PARAM_SOLVE_GROUPS, groups)
        out = run_problem(h, p, prec, max_refine=30, tol=1e-14, nb=nb)
    finally:
        g.rmat_destroy(h)
    assert out["status"] == g.RMAT_OK
    for k in ("U", "R", "X"):
        e = relerr(out[k], ref[k])
        assert e < TOL[prec], (k, e)


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("la,la_ctas,both", [(0, 0, 1), (1, 0, 1), (1, 1, 1), (1, 0, 1 << 30),
                                             (2, 0, 1)])
@pytest.mark.parametrize("nb,shape", [(64, (16, 100)), (128, (16, 100)), (128, (29, 50))])
def test_factor_lookahead_vs_oracle(g, prec, la, la_ctas, both, nb, shape):
    """RMAT_PARAM_FACTOR_LOOKAHEAD: each pair's far update split into the next pair's
    2 nb columns and the rest (side stream), the next pair's panels (as 32-column
    sub-panels with interchanges, U12 and updates between them), U12 on the second
    panel's columns and its column update beside the far part, the far columns' and
    earlier L columns' interchanges after it.  One look-ahead CTA puts the sub-panel's
    rows in global memory (up to 1536 rows of 32 columns at N = 1600); both = 2^30
    keeps only the first panel beside the far update; la = 2 issues the same order on
    one stream; with block width 128, N = 1450 ends in a 42-row block.  Same
    tolerances, all paths."""
    import torch
    torch.cuda.set_device(0)
    nch, nlag = shape
    p = cp.config3(16) if shape == (16, 100) else cp.make_problem(900 + nch, nch, nlag, 11.0)
    ref = truth(p, "c3-16" if shape == (16, 100) else ("steps", nch, nlag))
    h = g.rmat_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        g.rmat_set_param(h, g.RMAT_PARAM_FACTOR_LOOKAHEAD, la)
        g.rmat_set_param(h, g.RMAT_PARAM_LA_PANEL_CTAS, la_ctas)
        g.rmat_set_param(h, g.RMAT_PARAM_LA_MIN_ROWS, 1)  # look ahead at every pair
        g.rmat_set_param(h, g.RMAT_PARAM_LA_BOTH_ROWS, both)
        out = run_problem(h, p, prec, max_refine=30, tol=1e-14, nb=nb)
    finally:
        g.rmat_destroy(h)
    assert out["status"] == g.RMAT_OK
    assert out["info"] == 0
    for k in ("U", "R", "X"):
        e = relerr(out[k], ref[k])
        assert e < TOL[prec], (k, e)


@pytest.mark.parametrize("prec", PRECS)
def test_refinement_stops_at_fp64_floor(g, ctx, prec):
    """The refinement ends with RMAT_OK at the FP64 floor: once the normwise backward
    error max|r| / (max|C||X| + max|Phi|) is at most u/2 (u = 2^-53; the correctly
    rounded solution itself sits at 0.1-0.2 u on this family, measured by the oracle)
    one last correction is applied and no confirming residual is formed.  X, R, U are
    then at the truth's bounds."""
    p = cp.config3(16)
    ref = truth(p, "c3-16")
    out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14)
    berr = g.rmat_get_stats(ctx)["backward_error"]
    u = 2.0 ** -53
    assert out["status"] == g.RMAT_OK, (out["status"], berr / u)
    assert berr <= 0.5 * u
    hist = g.rmat_refine_history(ctx)
    assert len(hist) == out["iters"]
    for k in ("U", "R", "X"):
        assert relerr(out[k], ref[k]) < TOL[prec], k


def test_refinement_reports_stagnation_above_floor(g, ctx):
    """kappa = 1e10 with complex64 factors: classical refinement stalls far above the
    FP64 floor and says so (RMAT_ENOCONV, backward error > 2u)."""
    A, B, _ = cp.prescribed_kappa_hermitian(7, 512, 1e10, nrhs=3)
    out = run_dense(ctx, A, B, 2, max_refine=20, tol=1e-14)
    berr = g.rmat_get_stats(ctx)["backward_error"]
    assert out["status"] == g.RMAT_ENOCONV
    assert berr > 2.0 * 2.0 ** -53


@pytest.mark.parametrize("prec", [3, 1])
@pytest.mark.parametrize("blk", [128, 256])
@pytest.mark.parametrize("shape", [(16, 100), (29, 50)])
def test_solve_step_rows(g, ctx, prec, blk, shape):
    """Tensor-path solves in 128-row steps, or in 256-row steps over pairs of diagonal
    blocks (inverses composed from the 128-row ones): N = 1600 is six pairs and a
    64-row tail, N = 1450 five pairs, one unpaired full block and a 42-row tail."""
    nch, nlag = shape
    p = cp.make_problem(900 + nch, nch, nlag, 11.0)
    ref = truth(p, ("steps", nch, nlag))
    g.rmat_set_param(ctx, g.RMAT_PARAM_SOLVE_BLOCK, blk)
    try:
        out = run_problem(ctx, p, prec, max_refine=30, tol=1e-14, nb=128)
    finally:
        g.rmat_set_param(ctx, g.RMAT_PARAM_SOLVE_BLOCK, 0)
    assert out["status"] == g.RMAT_OK
    for k in ("X", "R", "U"):
        assert relerr(out[k], ref[k]) < TOL[prec], k
