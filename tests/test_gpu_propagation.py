"""R-matrix propagation over radial sectors on the GPU (-m gpu): U and R from
rmat_propagate against the oracle's propagation on the same sectors and mesh,
element by element; one sector against the single-system path; argument errors.
"""
import numpy as np
import pytest

import cc_problems as cp
from oracle import propagation as P
from rmat_gpu import relerr

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


def sector_potentials(g, p, radii):
    import torch
    Vs = []
    for s in range(len(radii) - 1):
        r = (g.rmat_mesh(p.nlag, radii[1])["r"] if s == 0
             else g.rmat_sector_mesh(p.nlag, radii[s], radii[s + 1])["r"])
        Vs.append(torch.from_numpy(cp.potential_at(p, r).ravel()).cuda())
    return Vs


def run_prop(g, ctx, p, radii, prec):
    import torch
    Vs = sector_potentials(g, p, radii)
    prob, keep = g.make_problem_struct(p.nch, p.nlag, radii[-1], p.hm, p.l, p.thresh, prec,
                                       zz=p.zz)
    no = int(np.sum(p.E - np.asarray(p.thresh) > 0))
    R = torch.zeros(p.nch * p.nch, dtype=torch.complex128, device="cuda")
    U = torch.zeros(max(no, 1) ** 2, dtype=torch.complex128, device="cuda")
    st, nopen = g.rmat_propagate(ctx, prob, p.E, radii, [v.data_ptr() for v in Vs],
                                 max_refine=30, tol=1e-14, R_dev=R.data_ptr(), U_dev=U.data_ptr())
    torch.cuda.synchronize()
    return (R.cpu().numpy().reshape(p.nch, p.nch).T,
            U.cpu().numpy()[:nopen * nopen].reshape(nopen, nopen).T, nopen)


CASES = {
    "neutral-3": (lambda: cp.make_problem(21, 3, 40, 10.0), [0.0, 7.5, 15.0]),
    "neutral-closed": (lambda: _closed(), [0.0, 5.0, 10.0, 15.0]),
    "charged-4": (lambda: cp.charged_problem(23, 4, 48, 30.0), [0.0, 8.0, 16.0, 24.0]),
}


def _closed():
    p = cp.make_problem(24, 4, 36, 6.0)
    p.thresh = np.array([0.0, 1.0, 2.5, 7.0])
    return p


def fp64_floor(p, radii):
    """Error of the propagated R and U when every sector is solved by a plain FP64
    LU (oracle, no refinement) against the double-double-refined truth: the FP64
    floor of the chained propagation and matching on this case."""
    pot = lambda r: cp.potential_at(p, r)  # noqa: E731
    U_t, R_t, _ = P.propagated_collision(p, radii, pot)
    U_0, R_0, _ = P.propagated_collision(p, radii, pot, refine_steps=0)
    return relerr(R_0, R_t), relerr(U_0, U_t)


@pytest.mark.parametrize("prec", [0, 3, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_propagation_matches_oracle(g, ctx, case, prec):
    make, radii = CASES[case]
    p = make()
    U_ref, R_ref, no = P.propagated_collision(p, radii, lambda r: cp.potential_at(p, r))
    R, U, nopen = run_prop(g, ctx, p, radii, prec)
    assert nopen == no
    eR, eU = relerr(R, R_ref), relerr(U, U_ref)
    if prec == 0:
        # FP64 path: each sector refined to its FP64 floor, then ns - 1 FP64 propagation
        # steps and the matching, whose rounding no refinement removes.  The bound is
        # twice the error of the same chain with plain FP64 LU sector solves (measured
        # by the oracle on this case: R 6e-13..2.2e-12, U 1.5e-12..2.3e-12), and never
        # below the single-system 1e-12
        fR, fU = fp64_floor(p, radii)
        print(f"{case} FP64: R {eR:.2e} (floor {fR:.2e}), U {eU:.2e} (floor {fU:.2e})")
        assert eR < max(1e-12, 2.0 * fR)
        assert eU < max(1e-12, 2.0 * fU)
    else:
        assert eR < TOL[prec]
        assert eU < TOL[prec]


def test_one_sector_equals_single_system(g, ctx):
    from rmat_gpu import run_problem
    p = cp.config1()
    R, U, _ = run_prop(g, ctx, p, [0.0, p.a], 0)
    out = run_problem(ctx, p, 0, max_refine=30, tol=1e-14)
    assert relerr(U, out["U"]) < 1e-13
    assert relerr(R, out["R"]) < 1e-13


def test_propagation_argument_errors(g, ctx):
    import torch
    p = cp.make_problem(25, 2, 20, 10.0)
    radii = [0.0, 5.0, 10.0]
    Vs = sector_potentials(g, p, radii)
    ptrs = [v.data_ptr() for v in Vs]
    U = torch.zeros(4, dtype=torch.complex128, device="cuda")
    bad_b, kb = g.make_problem_struct(p.nch, p.nlag, 10.0, p.hm, p.l, p.thresh, 0, bloch_B=-1.0)
    with pytest.raises(g.RmatError) as ei:
        g.rmat_propagate(ctx, bad_b, p.E, radii, ptrs, U_dev=U.data_ptr())
    assert ei.value.status == -2
    prob, keep = g.make_problem_struct(p.nch, p.nlag, 10.0, p.hm, p.l, p.thresh, 0)
    with pytest.raises(g.RmatError) as ei:
        g.rmat_propagate(ctx, prob, p.E, [0.0, 6.0, 5.0], ptrs, U_dev=U.data_ptr())
    assert ei.value.status == -3
    g.rmat_propagate(ctx, prob, p.E, radii, ptrs, U_dev=U.data_ptr())
    R = torch.zeros(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(g.RmatError) as ei:                 # no solved single system left
        g.rmat_collision(ctx, R.data_ptr(), U.data_ptr())
    assert ei.value.status == g.RMAT_ESTATE


@pytest.mark.parametrize("prec", [3, 0])
def test_concurrent_sectors_equal_sequential(g, ctx, prec):
    """Sectors on worker contexts (own streams and host threads) give the same R
    and U as one after the other on the caller's context (solve look-ahead off on the
    caller, as on the workers: its concurrent reduce-adds would vary the last bits
    from run to run)."""
    p = cp.charged_problem(27, 4, 48, 25.0)
    radii = [0.0, 6.0, 12.0, 18.0, 24.0]
    g.rmat_set_param(ctx, g.RMAT_PARAM_SOLVE_LOOKAHEAD, 0)
    try:
        g.rmat_set_param(ctx, g.RMAT_PARAM_PROP_CONCURRENT, 0)
        R0, U0, _ = run_prop(g, ctx, p, radii, prec)
        g.rmat_set_param(ctx, g.RMAT_PARAM_PROP_CONCURRENT, 1)
        R1, U1, _ = run_prop(g, ctx, p, radii, prec)
        R2, U2, _ = run_prop(g, ctx, p, radii, prec)      # workers reused
    finally:
        g.rmat_set_param(ctx, g.RMAT_PARAM_SOLVE_LOOKAHEAD, 1)
    assert relerr(U1, U0) < 1e-14 and relerr(R1, R0) < 1e-14
    assert relerr(U2, U1) < 1e-14
