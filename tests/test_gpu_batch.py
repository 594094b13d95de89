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
    # the small-system class (one persistent launch): one channel, all channels
    # closed but one, a charged pair below the barrier, the largest that fits
    out.append(cp.make_problem(602, 1, 100, 6.0))
    r = cp.make_problem(603, 4, 40, 3.0)
    r.thresh = np.array([0.0, 3.5, 4.0, 4.5])
    out.append(r)
    out.append(cp.charged_problem(604, 2, 50, 14.0))
    out.append(cp.make_problem(605, 4, 40, 22.0))
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
    run_batch(g, cases, prec, {g.RMAT_BATCH_LANES: lanes, g.RMAT_BATCH_SPLIT_N: split,
                               g.RMAT_BATCH_GRAPH: graph}, expect_graph=graph)


@pytest.mark.parametrize("prec", [3, 0])
@pytest.mark.parametrize("small", [0, -1])
def test_small_system_class(g, cases, prec, small):
    """The systems that fit one thread block (N <= 160 complex64, 112 complex128) in the
    persistent launch (-1) or through the lanes (0): same U against the oracle."""
    info = run_batch(g, cases, prec, {g.RMAT_BATCH_LANES: 4, g.RMAT_BATCH_SPLIT_N: 8192,
                                      g.RMAT_BATCH_SMALL_N: small})
    assert (info["small_systems"] > 0) == (small != 0)


@pytest.mark.parametrize("prec", [3])
def test_tile_shapes_and_tuner(g, cases, prec, tmp_path, monkeypatch):
    """128-wide tensor-update tiles and 64-wide LU blocks in the lanes, then the
    autotuner's plan (cached in RMAT_TUNE_CACHE): U against the oracle each time."""
    run_batch(g, cases, prec, {g.RMAT_BATCH_LANES: 4, g.RMAT_BATCH_SPLIT_N: 8192,
                               g.RMAT_BATCH_TC_BN: 128, g.RMAT_BATCH_NB_LANE: 64,
                               g.RMAT_BATCH_NB_SERIAL: 32})
    monkeypatch.setenv("RMAT_TUNE_CACHE", str(tmp_path / "tune.jsonl"))
    info = run_batch(g, cases, prec, {}, tune=True)
    assert (tmp_path / "tune.jsonl").read_text().count("nb_serial") == 1
    info2 = run_batch(g, cases, prec, {}, tune=True)          # from the cache
    for k in ("lanes", "split_n", "small_n", "nb_lane", "nb_serial", "tc_bn_lane"):
        assert info2[k] == info[k], k


def run_batch(g, cases, prec, settings, expect_graph=1, tune=False):
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
            for key, v in settings.items():
                g.rmat_batch_set(b, key, v)
            nopen = g.rmat_batch_nopen(b, len(probs))
            Us = [torch.zeros(max(1, n) ** 2, dtype=torch.complex128, device="cuda") for n in nopen]
            torch.cuda.synchronize()
            if tune:
                g.rmat_batch_tune(b, [u.data_ptr() for u in Us])
            for rep in range(2):                   # second run replays the graph
                st, it = g.rmat_batch_run(b, [u.data_ptr() for u in Us])
                torch.cuda.synchronize()
                for k, (p, ref) in enumerate(zip(probs, refs)):
                    assert nopen[k] == ref["nopen"]
                    assert st[k] == g.RMAT_OK, (k, st[k])   # every system reaches the floor
                    n = nopen[k]
                    if n == 0:
                        continue
                    U = Us[k].cpu().numpy()[:n * n].reshape(n, n).T
                    assert relerr(U, ref["U"]) < TOL[prec], (rep, k, relerr(U, ref["U"]))
            info = g.rmat_batch_info(b)
            assert info["systems"] == len(probs)
            assert info["graph"] == (1 if expect_graph else 0)
            return info
        finally:
            g.rmat_batch_destroy(b)
    finally:
        g.rmat_destroy(ctx)
