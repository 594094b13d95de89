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


def channel_blocks(p, V, mesh=None, T0=None) -> np.ndarray:
    """Kb[al] = the diagonal channel block C[(al,.),(al,.)] of the dense C, (nch, nlag, nlag).

    Entry for entry the numbers assemble_dense stores: hm T0 - hm (B/a) f f^T
    off the diagonal, fl(K_ii + fl(d_al,i + V_alal(r_i))) on it."""
    nch, nlag = p.nch, p.nlag
    m = mesh if mesh is not None else lagrange_mesh(nlag, p.a)
    T = T0 if T0 is not None else kinetic_bloch(nlag, p.a, m)
    f_a = m["f_a"]
    K = p.hm * T - p.hm * (p.bloch_B / p.a) * np.outer(f_a, f_a)
    d = channel_diagonal(p, m)
    Kb = np.broadcast_to(K.astype(np.complex128), (nch, nlag, nlag)).copy()
    ii = np.arange(nlag)
    for al in range(nch):
        Kb[al, ii, ii] = K[ii, ii] + (d[al] + V[al, al, :])
    return Kb


def structured_residual_dd(p, V, X, Phi=None, mesh=None, T0=None):
    """r = Phi - C X with C applied through its block structure, every product and
    every sum of C X accumulated in double-double (oracle.ddarith), rounded once.

    The structure is that of Eq. (block_structure) (Sec. 2): per row (al, i)
      (C X)[(al,i),be] = sum_j Kb[al][i,j] X[(al,j),be]
                       + sum_{al' != al} V_{al al'}(r_i) X[(al',i),be],
    Kb the diagonal channel blocks exactly as the dense C stores them
    (channel_blocks).  This is the residual of the paper's refinement (Sec. 3.2,
    Sec. 3.4 step 7) in extended precision, for the "truth" solution at sizes
    where the dense double-double residual (ddarith.dd_residual, O(N^2 nrhs)
    Python-level work) is out of reach.  Columns are independent: callers may
    evaluate any subset of columns of X (and Phi) separately.

    Pins (tests/test_oracle_system.py): equals ddarith.dd_residual of the dense C
    (itself pinned to exact rational arithmetic) to the last bit, and a dropped
    coupling or kinetic term is caught.
    """
    from .ddarith import dd_add, two_prod
    nch, nlag = p.nch, p.nlag
    m = mesh if mesh is not None else lagrange_mesh(nlag, p.a)
    B = Phi if Phi is not None else surface_rhs(p, m)
    nrhs = X.shape[1]
    X3 = X.reshape(nch, nlag, nrhs)
    Xr, Xi = np.ascontiguousarray(X3.real), np.ascontiguousarray(X3.imag)
    Kb = channel_blocks(p, V, m, T0)
    shape = (nch, nlag, nrhs)
    hr, lr = np.zeros(shape), np.zeros(shape)
    hi, li = np.zeros(shape), np.zeros(shape)

    def acc(h, l, a, b, sign):
        s, e = two_prod(a, b)
        return dd_add(h, l, sign * s, sign * e)

    # channel blocks: sum over j of Kb[al][i, j] X[(al, j), be]
    for j in range(nlag):
        kr = Kb[:, :, j].real[:, :, None]                 # [al, i, 1]
        ki = Kb[:, :, j].imag[:, :, None]
        xr = Xr[:, j, :][:, None, :]                      # [al, 1, be]
        xi = Xi[:, j, :][:, None, :]
        hr, lr = acc(hr, lr, kr, xr, 1.0)
        hr, lr = acc(hr, lr, ki, xi, -1.0)
        hi, li = acc(hi, li, kr, xi, 1.0)
        hi, li = acc(hi, li, ki, xr, 1.0)
    # point couplings: sum over al' != al of V_{al al'}(r_i) X[(al', i), be]
    for alp in range(nch):
        w = V[alp, :, :].copy()                            # [al, i] = V_{al alp}(r_i)
        w[alp, :] = 0.0                                    # al' = al sits in Kb's diagonal
        wr = w.real[:, :, None]
        wi = w.imag[:, :, None]
        xr = Xr[alp][None, :, :]                           # [1, i, be]
        xi = Xi[alp][None, :, :]
        hr, lr = acc(hr, lr, wr, xr, 1.0)
        hr, lr = acc(hr, lr, wi, xi, -1.0)
        hi, li = acc(hi, li, wr, xi, 1.0)
        hi, li = acc(hi, li, wi, xr, 1.0)
    B3 = B.reshape(nch, nlag, nrhs)
    rr_h, rr_l = dd_add(B3.real, np.zeros(shape), -hr, -lr)
    ri_h, ri_l = dd_add(B3.imag, np.zeros(shape), -hi, -li)
    return ((rr_h + rr_l) + 1j * (ri_h + ri_l)).reshape(X.shape)
