"""The allocation-free collision entry point agrees with rmat_collision (-m gpu).

rmat_collision_noalloc serves callers that cannot allocate device memory when
they need U (a pool allocator owning the device, no device synchronisation
allowed, a fixed memory budget).  It takes a solution X the caller holds and
writes R and U with its scratch in a fixed device array.  Two calls in a row
must reproduce rmat_collision's R and U to the FP64 tolerance of the other
tests (1e-12 relative): the second call also checks that the scratch left by
the first one does not leak into the result.  This file is collected last.
"""
import numpy as np
import pytest

import cc_problems as cp
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
        for call in range(2):
            R2 = torch.full((p.nch * p.nch,), float("nan"), dtype=torch.complex128, device="cuda")
            U2 = torch.full((no * no,), float("nan"), dtype=torch.complex128, device="cuda")
            n2 = g.rmat_collision_noalloc(prob, p.E, fa.data_ptr(), X.data_ptr(), p.N,
                                          R2.data_ptr(), U2.data_ptr(), stream)
            torch.cuda.synchronize()
            assert n2 == no
            assert relerr(R2.cpu().numpy(), R1.cpu().numpy()) < 1e-12, call
            assert relerr(U2.cpu().numpy(), U1.cpu().numpy()) < 1e-12, call
    finally:
        g.rmat_destroy(ctx)


def test_collision_noalloc_rejects_too_many_channels():
    import paper_2512_11590_gb300 as g
    p = cp.make_problem(1, 65, 10, 10.0)
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, g.RMAT_C128)
    with pytest.raises(g.RmatError) as ei:
        g.rmat_collision_noalloc(prob, p.E, 1, 1, p.N, 0, 1)
    assert ei.value.status == -1
