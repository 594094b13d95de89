"""The allocation-free collision entry point agrees with rmat_collision (-m gpu).

rmat_collision_noalloc serves callers that cannot allocate device memory when
they need U (a pool allocator owning the device, no device synchronisation
allowed, a fixed memory budget).  It takes a solution X the caller holds and
writes R and U with its scratch in a fixed device array.  Two calls in a row
must reproduce rmat_collision's R and U to the FP64 tolerance of the other
tests (1e-12 relative): the second call also checks that the scratch left by
the first one does not leak into the result.  The same R and U are also checked
against the CPU oracle's contraction and matching of the same X.  The edge
cases: no R output, every channel closed (no U), and a failing call followed by
a good one (the status word is cleared on every call).  This file is collected
last.
"""
import numpy as np
import pytest

import cc_problems as cp
from oracle.collision import collision_matrix, r_matrix
from rmat_gpu import relerr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["config1", "closed-channels", "nch16", "charged"])
def test_collision_noalloc_matches_rmat_collision(case):
    import torch

    import paper_2512_11590_gb300 as g
    if case == "config1":
        p = cp.config1()
    elif case == "closed-channels":
        p = cp.config1()
        p.E = 3.0
        p.thresh = np.array([0.0, 1.0, 4.0, 4.5])
    elif case == "charged":
        p = cp.charged_problem(78, 6, 80, 14.0)       # sub-barrier Coulomb channels
        p.thresh[-1] = 17.0                           # one closed charged channel
    else:
        p = cp.make_problem(77, 16, 60, 6.0)          # thresholds U(0,5): several closed channels
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = g.rmat_create(0, stream)
    try:
        m = g.rmat_mesh(p.nlag, p.a)
        V = torch.from_numpy(cp.potential_at(p, m["r"]).ravel()).cuda()
        prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, g.RMAT_C128,
                                           zz=p.zz)
        g.rmat_assemble(ctx, prob, p.E, V.data_ptr())
        g.rmat_factor(ctx)
        X = torch.zeros((p.nch, p.N), dtype=torch.complex128, device="cuda")
        g.rmat_solve(ctx, X.data_ptr(), p.N, 5, 1e-14)
        no = int(np.sum(p.E - p.thresh > 0))
        R1 = torch.zeros(p.nch * p.nch, dtype=torch.complex128, device="cuda")
        U1 = torch.zeros(no * no, dtype=torch.complex128, device="cuda")
        assert g.rmat_collision(ctx, R1.data_ptr(), U1.data_ptr()) == no
        fa = torch.from_numpy(m["f_a"]).cuda()
        Xh = X.cpu().numpy().T
        R_or = r_matrix(p, Xh, m["f_a"])
        U_or, no_or = collision_matrix(p, R_or)
        assert no_or == no
        for call in range(2):
            R2 = torch.full((p.nch * p.nch,), float("nan"), dtype=torch.complex128, device="cuda")
            U2 = torch.full((no * no,), float("nan"), dtype=torch.complex128, device="cuda")
            n2 = g.rmat_collision_noalloc(prob, p.E, fa.data_ptr(), X.data_ptr(), p.N,
                                          R2.data_ptr(), U2.data_ptr(), stream)
            torch.cuda.synchronize()
            assert n2 == no
            assert relerr(R2.cpu().numpy(), R1.cpu().numpy()) < 1e-12, call
            assert relerr(U2.cpu().numpy(), U1.cpu().numpy()) < 1e-12, call
            R2h = R2.cpu().numpy().reshape(p.nch, p.nch).T
            U2h = U2.cpu().numpy().reshape(no, no).T
            assert relerr(R2h, R_or) < 1e-12, call
            assert relerr(U2h, U_or) < 1e-12, call
        # no R output requested: U alone
        U3 = torch.full((no * no,), float("nan"), dtype=torch.complex128, device="cuda")
        assert g.rmat_collision_noalloc(prob, p.E, fa.data_ptr(), X.data_ptr(), p.N, 0,
                                        U3.data_ptr(), stream) == no
        torch.cuda.synchronize()
        assert relerr(U3.cpu().numpy(), U1.cpu().numpy()) < 1e-12
    finally:
        g.rmat_destroy(ctx)


def test_collision_noalloc_all_channels_closed():
    """E below every threshold: no open channel, nopen = 0 and no U is written."""
    import torch

    import paper_2512_11590_gb300 as g
    p = cp.config1()
    p.thresh = np.array([12.0, 13.0, 14.0, 15.0])     # E = 10 MeV: all closed
    m = g.rmat_mesh(p.nlag, p.a)
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, g.RMAT_C128)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    fa = torch.from_numpy(m["f_a"]).cuda()
    rng = np.random.default_rng(5)
    Xh = rng.standard_normal((p.N, p.nch)) + 1j * rng.standard_normal((p.N, p.nch))
    X = torch.from_numpy(np.asfortranarray(Xh).ravel(order="F")).cuda()
    R = torch.zeros(p.nch * p.nch, dtype=torch.complex128, device="cuda")
    assert g.rmat_collision_noalloc(prob, p.E, fa.data_ptr(), X.data_ptr(), p.N, R.data_ptr(), 0,
                                    stream) == 0
    torch.cuda.synchronize()
    assert relerr(R.cpu().numpy().reshape(p.nch, p.nch).T, r_matrix(p, Xh, m["f_a"])) < 1e-13


def test_collision_noalloc_failure_then_success():
    """A channel function that cannot converge (eta ~ 3e5) reports RMAT_ECHANFN; the
    next valid call returns RMAT_OK with the oracle's U (status cleared per call)."""
    import torch

    import paper_2512_11590_gb300 as g
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    bad = cp.charged_problem(9, 1, 20, 10.0)
    bad.zz = np.array([1e7])
    mb = g.rmat_mesh(bad.nlag, bad.a)
    pb, kb = g.make_problem_struct(bad.nch, bad.nlag, bad.a, bad.hm, bad.l, bad.thresh,
                                   g.RMAT_C128, zz=bad.zz)
    fab = torch.from_numpy(mb["f_a"]).cuda()
    Xb = torch.ones(bad.N, dtype=torch.complex128, device="cuda")
    Ub = torch.zeros(1, dtype=torch.complex128, device="cuda")
    with pytest.raises(g.RmatError) as ei:
        g.rmat_collision_noalloc(pb, bad.E, fab.data_ptr(), Xb.data_ptr(), bad.N, 0,
                                 Ub.data_ptr(), stream)
    assert ei.value.status == g.RMAT_ECHANFN
    p = cp.config1()
    m = g.rmat_mesh(p.nlag, p.a)
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, g.RMAT_C128)
    fa = torch.from_numpy(m["f_a"]).cuda()
    rng = np.random.default_rng(6)
    Xh = (rng.standard_normal((p.N, p.nch)) + 1j * rng.standard_normal((p.N, p.nch))) * 1e-3
    X = torch.from_numpy(np.asfortranarray(Xh).ravel(order="F")).cuda()
    U = torch.zeros(p.nch * p.nch, dtype=torch.complex128, device="cuda")
    assert g.rmat_collision_noalloc(prob, p.E, fa.data_ptr(), X.data_ptr(), p.N, 0, U.data_ptr(),
                                    stream) == p.nch
    torch.cuda.synchronize()
    U_or, _ = collision_matrix(p, r_matrix(p, Xh, m["f_a"]))
    assert relerr(U.cpu().numpy().reshape(p.nch, p.nch).T, U_or) < 1e-12


def test_collision_noalloc_rejects_bad_arguments():
    import paper_2512_11590_gb300 as g
    p = cp.make_problem(1, 65, 10, 10.0)
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, g.RMAT_C128)
    with pytest.raises(g.RmatError) as ei:
        g.rmat_collision_noalloc(prob, p.E, 1, 1, p.N, 0, 1)
    assert ei.value.status == -1
    q = cp.config1()
    for thresh, B, E, want in ((np.array([0.0, np.nan, 1.0, 2.0]), 0.0, 10.0, -1),
                               (q.thresh, np.inf, 10.0, -1), (q.thresh, 0.0, np.inf, -2),
                               (q.thresh, 0.0, np.nan, -2)):
        prob, keep = g.make_problem_struct(q.nch, q.nlag, q.a, q.hm, q.l, thresh, g.RMAT_C128,
                                           bloch_B=B)
        with pytest.raises(g.RmatError) as ei:
            g.rmat_collision_noalloc(prob, E, 1, 1, q.N, 0, 1)
        assert ei.value.status == want
