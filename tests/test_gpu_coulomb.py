"""Charged channels on the GPU (-m gpu): the collision matrix with Coulomb
asymptotics through the C ABI, element by element against the oracle.

Inputs follow the charged-particle recipe of cc_problems.charged_problem
(alpha + 208Pb-like: hm = 20.9/3.925 MeV fm^2, Z1 Z2 e^2 = 236.16 MeV fm,
uniformly charged sphere inside the nucleus).  Cases: above the Coulomb
barrier with a closed channel (Steed's method at rho = ka and the closed-
channel continued fraction), below it (inward integration of G inside the
turning point), one channel at l = 20 across the paper's E_cm = 10-50 MeV
validation range, a pure Coulomb interior (U = 1), and the error paths
(zz < 0 rejected, a channel function that cannot converge reported as
RMAT_ECHANFN).  Tolerances: FP64 path 1e-11 on U (both sides are FP64 with
channel functions accurate to ~1e-12), refined FP32 paths 1e-10.
"""
import numpy as np
import pytest

import cc_problems as cp
from oracle import oracle_solve
from rmat_gpu import relerr, run_problem

pytestmark = pytest.mark.gpu

TOL_U = {0: 1e-11, 1: 1e-10, 3: 1e-10}


@pytest.fixture(scope="module")
def ctx():
    import torch

    import paper_2512_11590_gb300 as g
    torch.cuda.set_device(0)
    c = g.rmat_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    g.rmat_destroy(c)


def above_barrier():
    p = cp.charged_problem(31, 5, 120, 30.0)
    p.thresh = np.array([0.0, 1.0, 2.5, 4.0, 33.0])      # last channel closed
    return p


def below_barrier():
    p = cp.charged_problem(32, 4, 100, 12.0)
    p.thresh = np.array([0.0, 0.7, 1.9, 14.5])            # sub-barrier open + one closed
    return p


@pytest.mark.parametrize("prec", [0, 3, 1])
@pytest.mark.parametrize("make", [above_barrier, below_barrier])
def test_charged_collision_matches_oracle(ctx, prec, make):
    p = make()
    ref = oracle_solve(p, refine_steps=3)
    out = run_problem(ctx, p, prec, max_refine=30 if prec else 0, tol=1e-14 if prec else 0.0)
    assert out["nopen"] == ref["nopen"]
    assert relerr(out["R"], ref["R"]) < 1e-11
    assert np.max(np.abs(out["U"] - ref["U"])) < TOL_U[prec]


@pytest.mark.parametrize("E", [10.0, 20.0, 30.0, 50.0])
def test_single_channel_l20_energy_scan(ctx, E):
    p = cp.charged_problem(5, 1, 140, E)
    p.l = np.array([20], dtype=np.int32)
    ref = oracle_solve(p, refine_steps=3)
    out = run_problem(ctx, p, 0)
    assert abs(out["U"][0, 0] - ref["U"][0, 0]) < 1e-11
    assert abs(out["U"][0, 0]) <= 1.0 + 1e-12


def test_pure_coulomb_interior_identity(ctx):
    p = cp.charged_problem(7, 3, 100, 30.0, V0=0.0, W=0.0, Rc=0.0)
    p.s[:] = 0.0
    p.l = np.array([0, 2, 3], dtype=np.int32)
    p.thresh = np.array([0.0, 1.5, 34.0])
    for prec in (0, 3):
        out = run_problem(ctx, p, prec, max_refine=30 if prec else 0, tol=1e-14 if prec else 0.0)
        assert out["nopen"] == 2
        assert np.max(np.abs(out["U"] - np.eye(2))) < 1e-8


def test_negative_zz_rejected(ctx):
    import torch

    import paper_2512_11590_gb300 as g
    p = cp.charged_problem(9, 2, 20, 30.0)
    m = g.rmat_mesh(p.nlag, p.a)
    V = torch.from_numpy(cp.potential_at(p, m["r"]).ravel()).cuda()
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, 0,
                                       zz=np.array([236.16, -1.0]))
    with pytest.raises(g.RmatError) as ei:
        g.rmat_assemble(ctx, prob, p.E, V.data_ptr())
    assert ei.value.status == -2


def test_unconvergeable_channel_function_reported(ctx):
    """eta ~ 3e5: CF1 at the turning point needs more terms than its bound."""
    import torch

    import paper_2512_11590_gb300 as g
    p = cp.charged_problem(9, 1, 20, 10.0)
    p.zz = np.array([1e7])
    m = g.rmat_mesh(p.nlag, p.a)
    V = torch.from_numpy(cp.potential_at(p, m["r"]).ravel()).cuda()
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, 0, zz=p.zz)
    g.rmat_assemble(ctx, prob, p.E, V.data_ptr())
    g.rmat_factor(ctx)
    X = torch.zeros((p.nch, p.N), dtype=torch.complex128, device="cuda")
    g.rmat_solve(ctx, X.data_ptr(), p.N, 0, 0.0)
    R = torch.zeros(1, dtype=torch.complex128, device="cuda")
    U = torch.zeros(1, dtype=torch.complex128, device="cuda")
    with pytest.raises(g.RmatError) as ei:
        g.rmat_collision(ctx, R.data_ptr(), U.data_ptr())
    assert ei.value.status == g.RMAT_ECHANFN
