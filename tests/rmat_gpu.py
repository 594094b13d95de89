"""GPU-side helpers for the parity tests: run a problem through the C ABI."""
import numpy as np


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def nopen_of(p):
    return int(np.sum(p.E - np.asarray(p.thresh) > 0))


def run_problem(ctx, p, precision, max_refine=0, tol=0.0, nb=0, V=None):
    """assemble -> factor -> solve (+refine) -> collision; returns host arrays."""
    import torch

    import cc_problems as cp
    import paper_2512_11590_gb300 as g
    g.rmat_set_param(ctx, g.RMAT_PARAM_NB, nb)
    m = g.rmat_mesh(p.nlag, p.a)
    if V is None:
        V = cp.potential_at(p, m["r"])
    Vd = torch.from_numpy(np.ascontiguousarray(V).ravel()).cuda()
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, precision,
                                       p.bloch_B, zz=p.zz)
    g.rmat_assemble(ctx, prob, p.E, Vd.data_ptr())
    fs, info = g.rmat_factor(ctx)
    X = torch.zeros((p.nch, p.N), dtype=torch.complex128, device="cuda")   # column-major N x nch
    st, iters, rel = g.rmat_solve(ctx, X.data_ptr(), p.N, max_refine, tol)
    no = nopen_of(p)
    R = torch.zeros(p.nch * p.nch, dtype=torch.complex128, device="cuda")
    U = torch.zeros(max(no, 1) ** 2, dtype=torch.complex128, device="cuda")
    nopen = g.rmat_collision(ctx, R.data_ptr(), U.data_ptr())
    torch.cuda.synchronize()
    return {"X": X.cpu().numpy().T, "R": R.cpu().numpy().reshape(p.nch, p.nch).T,
            "U": U.cpu().numpy()[:nopen * nopen].reshape(nopen, nopen).T, "nopen": nopen,
            "status": st, "iters": iters, "rel": rel, "info": info}


def run_dense(ctx, A, B, precision, max_refine=0, tol=0.0, nb=0):
    import torch

    import paper_2512_11590_gb300 as g
    n, nrhs = B.shape
    g.rmat_set_param(ctx, g.RMAT_PARAM_NB, nb)
    Ad = torch.from_numpy(np.asfortranarray(A).ravel(order="F")).cuda()
    Bd = torch.from_numpy(np.asfortranarray(B).ravel(order="F")).cuda()
    g.rmat_load_dense(ctx, n, nrhs, Ad.data_ptr(), n, Bd.data_ptr(), n, precision)
    fs, info = g.rmat_factor(ctx)
    X = torch.zeros((nrhs, n), dtype=torch.complex128, device="cuda")
    if fs != g.RMAT_OK:
        return {"X": None, "status": None, "iters": 0, "rel": None, "info": info,
                "factor_status": fs}
    st, iters, rel = g.rmat_solve(ctx, X.data_ptr(), n, max_refine, tol)
    torch.cuda.synchronize()
    return {"X": X.cpu().numpy().T, "status": st, "iters": iters, "rel": rel, "info": info,
            "factor_status": fs}
