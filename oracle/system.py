"""Dense internal-region matrix C, surface right-hand sides Phi, residuals (oracle).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

Matrix of Eq. (block_structure) (Sec. 2), written in MeV:

  C[(al,i),(al,j)]  = hm*T0[i,j] - hm*(B/a) f_i(a) f_j(a)
                      + delta_ij * (hm*l_al(l_al+1)/r_i^2 + V_alal(r_i) + E_al - E)
  C[(al,i),(al',i)] = V_al al'(r_i)                     (al != al')
  all other entries 0,

with channel-major index (al, i) -> al*nlag + i (the paper's (alpha-1)*nlag + i
of its R-matrix formula in Sec. 3.1, 0-based here).  K_alpha of
Eq. (block_structure) is the kinetic + Bloch + centrifugal + threshold part;
D_{alpha alpha'} = diag(V(r_i)) by the Lagrange property (Sec. 2).  The
right-hand sides (Sec. 3.1 step 2): Phi[(al,i), be] = delta_{al be} f_i(a).

Pins: the structured residual equals the dense one (test_oracle_system); the
whole matrix is pinned through the physics invariants of the collision matrix
(zero potential -> U = 1, square-well phase shift, unitarity, channel-radius
invariance, ODE integration; test_oracle_physics).
"""
from __future__ import annotations

import numpy as np

from .mesh import kinetic_bloch, lagrange_mesh


def channel_diagonal(p, mesh) -> np.ndarray:
    """d[al, i] = hm l(l+1)/r_i^2 + E_al - E  (the potential's diagonal is added separately)."""
    r = mesh["r"]
    l = np.asarray(p.l, dtype=np.float64)
    return p.hm * (l * (l + 1.0))[:, None] / (r * r)[None, :] + (np.asarray(p.thresh) - p.E)[:, None]


def assemble_dense(p, V: np.ndarray, mesh=None, T0=None):
    """Return (C, Phi): C is (N, N) complex128, Phi is (N, nch) complex128.

    ``V`` is the potential at this mesh, shape (nch, nch, nlag) with
    V[c2, c1, i] = V_{c1 c2}(r_i) (see cc_problems.potential_at).
    """
    nch, nlag = p.nch, p.nlag
    m = mesh if mesh is not None else lagrange_mesh(nlag, p.a)
    T = T0 if T0 is not None else kinetic_bloch(nlag, p.a, m)
    f_a = m["f_a"]
    N = nch * nlag
    C = np.zeros((N, N), dtype=np.complex128)
    K = p.hm * T - p.hm * (p.bloch_B / p.a) * np.outer(f_a, f_a)
    d = channel_diagonal(p, m)
    for al in range(nch):
        blk = slice(al * nlag, (al + 1) * nlag)
        C[blk, blk] = K
        for i in range(nlag):
            C[al * nlag + i, al * nlag + i] += d[al, i] + V[al, al, i]
        for alp in range(nch):
            if alp == al:
                continue
            for i in range(nlag):
                C[al * nlag + i, alp * nlag + i] = V[alp, al, i]
    Phi = np.zeros((N, nch), dtype=np.complex128)
    for be in range(nch):
        Phi[be * nlag:(be + 1) * nlag, be] = f_a
    return C, Phi


def surface_rhs(p, mesh=None) -> np.ndarray:
    m = mesh if mesh is not None else lagrange_mesh(p.nlag, p.a)
    Phi = np.zeros((p.N, p.nch), dtype=np.complex128)
    for be in range(p.nch):
        Phi[be * p.nlag:(be + 1) * p.nlag, be] = m["f_a"]
    return Phi


def dense_residual(C, X, B):
    """r = B - C X in complex128 (plain matrix product)."""
    return B - C @ X


def structured_apply(p, V, X, mesh=None, T0=None):
    """y = C X using only the block structure of Eq. (block_structure).

    y[(al,i),be] = hm sum_j T0[i,j] X[(al,j),be] - hm (B/a) f_i(a) sum_j f_j(a) X[(al,j),be]
                   + (d[al,i] + V_alal(r_i)) X[(al,i),be]
                   + sum_{al' != al} V_{al al'}(r_i) X[(al',i),be].
    Never forms the N x N matrix: this is the residual the refinement of the
    paper's Type 2 / hybrid solvers needs (Sec. 3.2, 3.4), evaluated from
    O(nlag^2 + nlag nch^2) numbers instead of N^2.
    """
    nch, nlag = p.nch, p.nlag
    m = mesh if mesh is not None else lagrange_mesh(nlag, p.a)
    T = T0 if T0 is not None else kinetic_bloch(nlag, p.a, m)
    f_a = m["f_a"]
    X3 = X.reshape(nch, nlag, -1)                     # [al, i, be]
    K = p.hm * T - p.hm * (p.bloch_B / p.a) * np.outer(f_a, f_a)
    y = np.einsum("ij,ajb->aib", K, X3)
    d = channel_diagonal(p, m)
    y += d[:, :, None] * X3
    # full potential matrix per mesh point: W[i, al, al'] = V_{al al'}(r_i)
    Wm = np.transpose(V, (2, 1, 0))                   # [i, c1, c2] = V_{c1 c2}(r_i)
    y += np.einsum("iac,cib->aib", Wm, X3)
    return y.reshape(X.shape)


def structured_residual(p, V, X, Phi=None, mesh=None, T0=None):
    """r = Phi - C X with C applied through its block structure (complex128)."""
    B = Phi if Phi is not None else surface_rhs(p, mesh)
    return B - structured_apply(p, V, X, mesh, T0)
