"""Write tests/golden/truth_config3_W*_n25600.txt from the CPU oracle alone.

Config 3 at full size: nch=256, nlag=100 (N=25600), 256 right-hand sides,
a=15 fm, E=10 MeV, hm=20.9 MeV fm^2, complex Woods-Saxon V0=-50 with W=-10
(config 3) or W=-1 (config 3b), seeded couplings (seed 11592).

The truth solution is oracle.refine.truth_solve_structured: LAPACK zgetrf of the
dense complex128 C (the paper's Type-1 factorisation, Sec. 3.1) and two
corrections with the residual in double-double through C's block structure
(Sec. 3.2 refinement, oracle.system.structured_residual_dd), evaluated on column
chunks in parallel worker processes (the columns are independent).  R and U then
come from oracle.collision.  A full N x 256 X is 105 MB, so the files keep
seeded samples: X at 1024 (row, column) positions, R and U at 512 positions plus
their whole diagonals, and the maxima of |X|, |R|, |U| over all entries (the
denominators of the max|delta|/max|ref| error).  Run from the repo root
(about 10 minutes and 25 GB of host memory per case on 8 cores):
    python tests/golden/make_truth_n25600.py [W ...]
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SAMPLE_SEED = 25600
N_X, N_RU = 1024, 512
CHUNK = 16

_G = {}


def _init(p, V):
    sys.path.insert(0, ROOT)
    from oracle.mesh import kinetic_bloch, lagrange_mesh
    m = lagrange_mesh(p.nlag, p.a)
    _G.update(p=p, V=V, m=m, T0=kinetic_bloch(p.nlag, p.a, m))


def _chunk_residual(args):
    from oracle.system import structured_residual_dd
    X, Phi = args
    g = _G
    return structured_residual_dd(g["p"], g["V"], X, Phi, g["m"], g["T0"])


def sample_positions(nrow, ncol, n, rng):
    return rng.integers(0, nrow, size=n), rng.integers(0, ncol, size=n)


def truth_file(W):
    return os.path.join(HERE, f"truth_config3_W{W:g}_n25600.txt")


def make_case(W, pool_size):
    import cc_problems as cp
    from oracle.collision import collision_matrix, r_matrix
    from oracle.mesh import lagrange_mesh
    from oracle.refine import truth_solve_structured

    p = cp.config3(256, W=W)
    m = lagrange_mesh(p.nlag, p.a)
    V = cp.potential_at(p, m["r"])
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(pool_size, initializer=_init, initargs=(p, V)) as pool:
        holder = {}

        def residual(X):
            Phi = holder["Phi"]
            parts = [(np.ascontiguousarray(X[:, c:c + CHUNK]), np.ascontiguousarray(Phi[:, c:c + CHUNK]))
                     for c in range(0, X.shape[1], CHUNK)]
            return np.concatenate(pool.map(_chunk_residual, parts), axis=1)

        from oracle.system import surface_rhs
        holder["Phi"] = surface_rhs(p, m)
        X, hist, _ = truth_solve_structured(p, V, m, steps=2, residual=residual)
    R = r_matrix(p, X, m["f_a"])
    U, nopen = collision_matrix(p, R)
    rng = np.random.default_rng(SAMPLE_SEED)
    xi, xj = sample_positions(p.N, p.nch, N_X, rng)
    ri, rj = sample_positions(p.nch, p.nch, N_RU, rng)
    ui, uj = sample_positions(nopen, nopen, N_RU, rng)
    d = np.arange(p.nch)
    du = np.arange(nopen)
    lines = [
        f"# config3 W={W:g}: nch=256 nlag=100 N=25600, 256 rhs, seed {p.seed}; truth X, R, U "
        f"(LAPACK zgetrf + 2 double-double structured-residual corrections), written by "
        f"tests/golden/make_truth_n25600.py from the CPU oracle",
        f"# refinement history max|r|/max|Phi|: {' '.join(f'{h:.3e}' for h in hist)}",
        f"# wall {time.time() - t0:.0f} s",
        f"max X {np.max(np.abs(X)):.17e}",
        f"max R {np.max(np.abs(R)):.17e}",
        f"max U {np.max(np.abs(U)):.17e}",
        f"nopen {nopen}",
    ]
    for name, M, ii, jj in (("X", X, xi, xj), ("R", R, np.concatenate([ri, d]), np.concatenate([rj, d])),
                            ("U", U, np.concatenate([ui, du]), np.concatenate([uj, du]))):
        for a, b in zip(ii, jj):
            z = M[a, b]
            lines.append(f"{name} {a} {b} {z.real:.17e} {z.imag:.17e}")
    with open(truth_file(W), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"W={W:g}: history {hist}, wall {time.time() - t0:.0f} s", flush=True)


def load_truth(W):
    """{'max': {X, R, U}, 'nopen': int, 'X'|'R'|'U': (rows, cols, values)}"""
    out = {"max": {}, "nopen": None}
    rows = {"X": [], "R": [], "U": []}
    with open(truth_file(W)) as f:
        for line in f:
            if line.startswith("#"):
                continue
            t = line.split()
            if t[0] == "max":
                out["max"][t[1]] = float(t[2])
            elif t[0] == "nopen":
                out["nopen"] = int(t[1])
            else:
                rows[t[0]].append((int(t[1]), int(t[2]), float(t[3]) + 1j * float(t[4])))
    for k, v in rows.items():
        a = np.array([r[0] for r in v]), np.array([r[1] for r in v]), np.array([r[2] for r in v])
        out[k] = a
    return out


def sampled_relerr(M, truth, name):
    """max over the sampled entries of |M - truth| / max|truth| (max over all entries)."""
    i, j, v = truth[name]
    return float(np.max(np.abs(np.asarray(M)[i, j] - v)) / truth["max"][name])


if __name__ == "__main__":
    Ws = [float(w) for w in sys.argv[1:]] or [-10.0, -1.0]
    for W in Ws:
        make_case(W, min(8, os.cpu_count() or 1))
