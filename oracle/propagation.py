"""R-matrix propagation over radial sectors (oracle).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

The paper's interface takes ns sectors (hprmat_init(nr, ns, rmax, ...) and
hprmat_solve(..., nr, ns, cpot, ...), Sec. 4, language bindings): the internal
region (0, a) is cut at 0 = a_0 < a_1 < ... < a_ns = a and the R-matrix is
carried from sector to sector; the paper prints no formula.  This module writes
out the standard propagation with Lagrange meshes:

* sector 1, (0, a_1): the regularised basis and matrix of oracle.mesh /
  oracle.system; its R-matrix in length units is Rl_1 = a_1 R(a_1) = hm Phi^T X;
* sector s >= 2, (r1, r2) = (a_{s-1}, a_s), h = r2 - r1: the Lagrange-Legendre
  basis without regularisation, f_i(r) = l_i(x) / sqrt(h w_i), x = (r - r1)/h,
  l_i the Lagrange polynomial through the Gauss-Legendre nodes x_k of (0, 1)
  (weights w_k); f_i(r_j) = delta_ij / sqrt(h w_j) and f_i is non-zero at both
  ends.  With the Bloch operator L = delta(r - r2) d/dr - delta(r - r1) d/dr the
  kinetic + Bloch matrix is symmetric,
      K_ij = hm int_{r1}^{r2} f_i' f_j' dr
           = hm / (h^2 sqrt(w_i w_j)) sum_k w_k l_i'(x_k) l_j'(x_k)
  (exact: the integrand has degree 2n - 4), and the sector's equation
  (T + L + V - E) u = L u becomes C c = hm (phi_R u'(r2) - phi_L u'(r1)),
  phi_L, phi_R the boundary values f_i(r1), f_i(r2) per channel.  With
  g_ab = hm phi_a^T C^-1 phi_b (nch x nch blocks, a, b in {L, R}):
      u(r1) = g_LR u'(r2) - g_LL u'(r1),   u(r2) = g_RR u'(r2) - g_RL u'(r1),
  and u(r1) = Rl_{s-1} u'(r1) gives
      Rl_s = g_RR - g_RL (Rl_{s-1} + g_LL)^-1 g_LR;
* finally R(a) = Rl_ns / a and U as for one sector (oracle.collision) at a.

The sector systems are solved like oracle.pipeline's reference: LU plus
double-double refinement (oracle.refine.truth_solve).

l_i' at the nodes and l_i(0), l_i(1) come from the barycentric form of the
Lagrange polynomials, the barycentric weights 1/prod_{m != i}(x_i - x_m)
accumulated as logarithms (no under- or overflow at large n).

Pins (tests/test_oracle_propagation.py): the sector kinetic matrix against the
integral of products of explicitly evaluated derivative polynomials (numpy
polynomial fits), the Lagrange property and boundary values by direct
evaluation; a free sector carries the exact Riccati-Bessel log-derivative
(u = sin(kr)); U with 2 or 3 sectors equals U with one sector over the same
(0, a) to mesh accuracy and direct ODE integration.
"""
from __future__ import annotations

import numpy as np

from .collision import collision_matrix
from .lu import solve
from .refine import truth_solve
from .mesh import gauss_legendre_unit, kinetic_bloch, lagrange_mesh
from .system import assemble_dense


def _barycentric_log(x: np.ndarray):
    """log|beta_i| and sign(beta_i), beta_i = 1 / prod_{m != i} (x_i - x_m)."""
    n = x.size
    logb = np.zeros(n)
    sgn = np.ones(n)
    for i in range(n):
        d = x[i] - np.delete(x, i)
        logb[i] = -np.sum(np.log(np.abs(d)))
        sgn[i] = np.prod(np.sign(d))
    return logb, sgn


def _lagrange_at(x: np.ndarray, logb, sgn, t: float) -> np.ndarray:
    """l_i(t) for all i (t not a node), barycentric second form."""
    terms = sgn * np.exp(logb - logb.max()) / (t - x)
    return terms / terms.sum()


def _derivative_matrix(x: np.ndarray, logb, sgn) -> np.ndarray:
    """D[k, i] = l_i'(x_k)."""
    n = x.size
    D = np.zeros((n, n))
    for k in range(n):
        for i in range(n):
            if i != k:
                # (beta_i / beta_k) / (x_k - x_i)
                D[k, i] = sgn[i] * sgn[k] * np.exp(logb[i] - logb[k]) / (x[k] - x[i])
        D[k, k] = np.sum(1.0 / (x[k] - np.delete(x, k)))
    return D


def sector_mesh(nlag: int, r1: float, r2: float) -> dict:
    """Non-regularised Lagrange-Legendre mesh of the sector (r1, r2).

    Returns r (points), lam (weights h w), fL = f_i(r1), fR = f_i(r2) and
    Kf = int f_i' f_j' dr (fm^-2; times hm gives the kinetic + Bloch block)."""
    if not r2 > r1:
        raise ValueError("sector needs r2 > r1")
    h = r2 - r1
    x, _, w = gauss_legendre_unit(nlag)
    logb, sgn = _barycentric_log(x)
    D = _derivative_matrix(x, logb, sgn)
    s = 1.0 / np.sqrt(h * w)
    fL = _lagrange_at(x, logb, sgn, 0.0) * s
    fR = _lagrange_at(x, logb, sgn, 1.0) * s
    Kf = (D.T * w) @ D / (h * h * np.sqrt(np.outer(w, w)))
    return {"r": r1 + h * x, "lam": h * w, "fL": fL, "fR": fR, "Kf": Kf, "x": x, "w": w,
            "r1": float(r1), "r2": float(r2)}


def sector_matrix(p, V: np.ndarray, sm: dict) -> np.ndarray:
    """C of one sector: hm Kf per channel block + diag(hm l(l+1)/r^2 + E_al - E) + V."""
    nch, n = p.nch, sm["r"].size
    r = sm["r"]
    l = np.asarray(p.l, dtype=np.float64)
    C = np.zeros((nch * n, nch * n), dtype=np.complex128)
    for al in range(nch):
        blk = slice(al * n, (al + 1) * n)
        C[blk, blk] = p.hm * sm["Kf"]
        C[blk, blk] += np.diag(p.hm * l[al] * (l[al] + 1.0) / r ** 2 + p.thresh[al] - p.E)
        for alp in range(nch):
            C[al * n + np.arange(n), alp * n + np.arange(n)] += V[alp, al, :]
    return C


def sector_green(p, V: np.ndarray, sm: dict, refine_steps: int = 2):
    """(g_LL, g_LR, g_RL, g_RR), g_ab = hm phi_a^T C^-1 phi_b, nch x nch.

    refine_steps = 0 gives the plain FP64 LU solve (no refinement)."""
    nch, n = p.nch, sm["r"].size
    C = sector_matrix(p, V, sm)
    Phi = np.zeros((nch * n, 2 * nch), dtype=np.complex128)
    for al in range(nch):
        Phi[al * n:(al + 1) * n, al] = sm["fL"]
        Phi[al * n:(al + 1) * n, nch + al] = sm["fR"]
    X, _ = truth_solve(C, Phi, steps=refine_steps)
    G = p.hm * (Phi.T @ X)
    return G[:nch, :nch], G[:nch, nch:], G[nch:, :nch], G[nch:, nch:]


def propagate(Rl: np.ndarray, g) -> np.ndarray:
    """Rl_s = g_RR - g_RL (Rl_{s-1} + g_LL)^-1 g_LR."""
    gLL, gLR, gRL, gRR = g
    return gRR - gRL @ solve(Rl + gLL, gLR)


def propagated_collision(p, radii, potential, refine_steps: int = 2):
    """U (and R at a = radii[-1]) with sectors (radii[s-1], radii[s]), nlag points each.

    potential(r) -> V array [c2, c1, i] at radii r (cc_problems.potential_at layout).
    refine_steps: double-double refinement steps of every sector solve (2: the truth;
    0: plain FP64 LU solves, which measures the FP64 floor of the propagated R, U)."""
    import copy
    radii = [float(v) for v in radii]
    q = copy.copy(p)
    q.a = radii[1]
    m = lagrange_mesh(p.nlag, q.a)
    T0 = kinetic_bloch(p.nlag, q.a, m)
    C, Phi = assemble_dense(q, potential(m["r"]), m, T0)
    X, _ = truth_solve(C, Phi, steps=refine_steps)
    Rl = p.hm * (Phi.T @ X)                      # = a_1 R(a_1)
    for s in range(2, len(radii)):
        sm = sector_mesh(p.nlag, radii[s - 1], radii[s])
        Rl = propagate(Rl, sector_green(p, potential(sm["r"]), sm, refine_steps))
    q.a = radii[-1]
    R = Rl / q.a
    U, nopen = collision_matrix(q, R)
    return U, R, nopen
