"""Batched systems (a11) on the GPU: every system's U against the CPU oracle,
and the batch against the per-system path (-m gpu)."""
import numpy as np
import pytest

import cc_problems as cp
from oracle import oracle_solve
from rmat_gpu import relerr, run_problem

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10, 2: 1e-10, 3: 1e-10}


def mixed_problems():
    """Small and medium systems of the config-4 family, including closed channels."""
    out = []
    for k, (nch, nlag, E) in enumerate([(2, 40, 3.0), (4, 60, 12.0), (2, 100, 30.0), (8, 40, 2.5),
                                         (4, 100, 45.0), (8, 80, 9.0), (16, 40, 20.0),
                                         (16, 100, 7.0), (3, 37, 15.0)]):
        out.append(cp.make_problem(500 + k, nch, nlag, E))
    # charged channels: above the Coulomb barrier with a closed channel, and below it
    q = cp.charged_problem(600, 4, 80, 25.0)
    q.thresh = np.array([0.0, 2.0, 3.5, 27.0])
    out.append(q)
    out.append(cp.charged_problem(601, 2, 100, 12.0))
    return out


@pytest.fixture(scope="module")
def cases():
    probs = mixed_problems()
    return probs, [oracle_solve(p, refine_steps=3) for p in probs]


@pytest.fixture(scope="module")
def g():
    import paper_2512_11590_gb300 as mod
    mod.lib()
    return mod


@pytest.mark.parametrize("prec", [3, 1, 0])
@pytest.mark.parametrize("lanes,split,graph", [(0, 0, 1), (4, 832, 1), (4, 832, 0), (8, 8192, 1)])
def test_batch_matches_oracle(g, cases, prec, lanes, split, graph):
    import torch
    torch.cuda.set_device(0)
    probs, refs = cases
    stream = torch.cuda.Stream()                 # a capturable (non-default) stream
    ctx = g.rmat_create(0, stream.cuda_stream)
    try:
        Vs, structs, keep = [], [], []
        for p in probs:
            m = g.rmat_mesh(p.nlag, p.a)
            Vs.append(torch.from_numpy(cp.potential_at(p, m["r"]).ravel()).cuda())
            s, k = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, prec,
                                            p.bloch_B, zz=p.zz)
            structs.append(s)
            keep.append(k)
        b = g.rmat_batch_create(ctx, structs, [p.E for p in probs], [v.data_ptr() for v in Vs],
                                max_refine=30, tol=1e-14)
        try:
            g.rmat_batch_set(b, g.RMAT_BATCH_LANES, lanes)
            g.rmat_batch_set(b, g.RMAT_BATCH_SPLIT_N, split)
            g.rmat_batch_set(b, g.RMAT_BATCH_GRAPH, graph)
            nopen = g.rmat_batch_nopen(b, len(probs))
            Us = [torch.zeros(max(1, n) ** 2, dtype=torch.complex128, device="cuda") for n in nopen]
            torch.cuda.synchronize()
            for rep in range(2):                   # second run replays the graph
                st, it = g.rmat_batch_run(b, [u.data_ptr() for u in Us])
                torch.cuda.synchronize()
                for k, (p, ref) in enumerate(zip(probs, refs)):
                    assert nopen[k] == ref["nopen"]
                    assert st[k] in (g.RMAT_OK, g.RMAT_ENOCONV), (k, st[k])
                    n = nopen[k]
                    if n == 0:
                        continue
                    U = Us[k].cpu().numpy()[:n * n].reshape(n, n).T
                    assert relerr(U, ref["U"]) < TOL[prec], (rep, k, relerr(U, ref["U"]))
            info = g.rmat_batch_info(b)
            assert info["systems"] == len(probs)
            assert info["graph"] == (1 if graph else 0)
        finally:
            g.rmat_batch_destroy(b)
    finally:
        g.rmat_destroy(ctx)
