"""The FP64 refinement residual r = Phi - C X on the GPU (-m gpu), through rmat_residual.

Every product mode (RMAT_PARAM_RESIDUAL = 1: point couplings on the FP64 tensor
instruction; = 2: point couplings as integer digit products on the FP16 tensor cores;
= 3: the kinetic part that way too) is compared element by element with the oracle's
double-double structured residual of the same X.  The
bound is the rounding of an FP64 evaluation, 16 u max(|C||X|) (u = 2^-53; a sum
of nlag + nch products rounds to ~sqrt(nlag + nch) u of its terms), for modes 1
and 2, and the digit cut of the kinetic rows for mode 3 (bound_for), checked on
the truth solution (r cancels to ~1e-12 of Phi: the regime the refinement works
in) and on a random X, at sizes with ragged tiles (nch and nrhs not multiples of
the 128 x 64 tiles, K padded to 16).
"""
import numpy as np
import pytest

import cc_problems as cp
from oracle import mesh as M
from oracle import system as S
from oracle.refine import truth_solve_structured

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


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


CASES = {
    "nch40": lambda: cp.make_problem(41, 40, 30, 12.0),
    "config3-nch64": lambda: cp.config3(64),
    "charged-nch33": lambda: cp.charged_problem(43, 33, 40, 25.0),
    "nch5": lambda: cp.make_problem(44, 5, 37, 9.0),
}


def bound_for(mode, nlag):
    """Error bound in u max|C||X|: FP64 rounding (16 u) for the FP64 products and the
    digit products of the couplings; for the digit product of the kinetic part
    (mode 3) the cut of each row of K at 2^-54 of its largest (diagonal) entry and of
    X at 2^-54 of its column maximum, summed over nlag terms: up to ~nlag/2 u."""
    return 16.0 if mode in (1, 2) else max(16.0, 0.5 * nlag)


def gpu_residual(g, ctx, p, X, mode):
    import torch
    g.rmat_set_param(ctx, g.RMAT_PARAM_RESIDUAL, mode)
    m = g.rmat_mesh(p.nlag, p.a)
    V = torch.from_numpy(cp.potential_at(p, m["r"]).ravel()).cuda()
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, g.RMAT_C128,
                                       zz=p.zz)
    g.rmat_assemble(ctx, prob, p.E, V.data_ptr())
    Xd = torch.from_numpy(np.asfortranarray(X).ravel(order="F")).cuda()
    Rd = torch.zeros_like(Xd)
    g.rmat_residual(ctx, Xd.data_ptr(), p.N, Rd.data_ptr(), p.N)
    torch.cuda.synchronize()
    return Rd.cpu().numpy().reshape(p.nch, p.N).T


@pytest.mark.parametrize("which", ["truth", "random"])
@pytest.mark.parametrize("case", list(CASES))
def test_residual_matches_double_double(g, ctx, case, which):
    p = CASES[case]()
    m = M.lagrange_mesh(p.nlag, p.a)
    V = cp.potential_at(p, m["r"])
    if which == "truth":
        X, _, Phi = truth_solve_structured(p, V, m, steps=2)
    else:
        rng = np.random.default_rng(7)
        X = rng.standard_normal((p.N, p.nch)) + 1j * rng.standard_normal((p.N, p.nch))
        Phi = S.surface_rhs(p, m)
    r_dd = S.structured_residual_dd(p, V, X, Phi, m)
    C, _ = S.assemble_dense(p, V, m)
    scale = np.max(np.abs(C) @ np.abs(X))
    for mode in (1, 2, 3):
        r = gpu_residual(g, ctx, p, X, mode)
        err = np.max(np.abs(r - r_dd)) / (U64 * scale)
        print(f"{case} {which} mode {mode}: max|r - r_dd| = {err:.2f} u max|C||X|")
        assert err < bound_for(mode, p.nlag), (mode, err)


def test_residual_modes_agree_on_the_bench_family(g, ctx):
    """config-3 family at nch = 128 (two 128-row tiles, K = 128): the tensor-core and
    FP64-instruction products agree within the FP64 rounding bound."""
    p = cp.config3(128)
    rng = np.random.default_rng(8)
    X = (rng.standard_normal((p.N, p.nch)) + 1j * rng.standard_normal((p.N, p.nch))) * 1e-3
    r1 = gpu_residual(g, ctx, p, X, 1)
    r2 = gpu_residual(g, ctx, p, X, 2)
    r3 = gpu_residual(g, ctx, p, X, 3)
    m = M.lagrange_mesh(p.nlag, p.a)
    V = cp.potential_at(p, m["r"])
    Kb = S.channel_blocks(p, V, m)
    # max |C||X| through the structure (the dense C would be 2.6 GB here)
    X3 = np.abs(X).reshape(p.nch, p.nlag, -1)
    absCX = np.einsum("aij,ajb->aib", np.abs(Kb), X3)
    Wabs = np.abs(np.transpose(V, (2, 1, 0)))
    for al in range(p.nch):
        Wabs[:, al, al] = 0.0
    absCX += np.einsum("iac,cib->aib", Wabs, X3)
    err = np.max(np.abs(r1 - r2)) / (U64 * np.max(absCX))
    err3 = np.max(np.abs(r1 - r3)) / (U64 * np.max(absCX))
    print(f"nch128: max|r_fp64mma - r_tensor| = {err:.2f}, kinetic too {err3:.2f} u max|C||X|")
    assert err < 16.0 and err3 < bound_for(3, p.nlag)


def test_residual_argument_errors(g, ctx):
    import torch
    X = torch.zeros(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(g.RmatError) as ei:              # nothing assembled yet
        g.rmat_residual(ctx, X.data_ptr(), 2, X.data_ptr(), 2)
    assert ei.value.status == g.RMAT_ESTATE
    with pytest.raises(g.RmatError) as ei:
        g.rmat_residual(ctx, 0, 2, X.data_ptr(), 2)
    assert ei.value.status == -2
    with pytest.raises(g.RmatError):
        g.rmat_set_param(ctx, g.RMAT_PARAM_RESIDUAL, 4)
