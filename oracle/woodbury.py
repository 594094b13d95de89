"""Woodbury-kinetic (Type 3) form of the internal-region system (oracle).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

Sec. 3.3 (Woodbury-kinetic solver) splits the matrix of Eq. (block_structure)
as M = K_diag + V_coupling, K_diag = I_nch (x) K with K the real kinetic +
Bloch matrix shared by every channel, and V_coupling everything of M that is
diagonal in the radial index (potential, centrifugal term, threshold, -E):

    V_{al al'}(r_j) = M[(al,j),(al',j)] - K[j,j] delta_{al al'}.

Then M c = b is the Schur-type system (I + K_diag^{-1} V_coupling) c = K_diag^{-1} b,
written in radial-major order (index (i, al) -> i*nch + al) as

    S[(i,al),(j,al')] = delta_ij delta_{al al'} + Kinv[i,j] V_{al al'}(r_j),
    b~[(i,al), be]    = sum_j Kinv[i,j] q2(r_j) delta_{al be},

whose solution, reordered to channel-major, is the solution X of M X = Phi.
K does not depend on E, so Kinv is formed once per mesh.

Pins (tests/test_oracle_woodbury.py): I_nch (x) K times S, reordered, gives back
the independently assembled M; the reordered solution of S equals the direct
solution of M X = Phi; S at two energies differs by -dE Kinv (x) I only; a
planted index mistake (V taken at r_i instead of r_j) is caught.
"""
from __future__ import annotations

import numpy as np

from .lu import solve
from .mesh import kinetic_bloch, lagrange_mesh
from .system import channel_diagonal


def kinetic_matrix(p, mesh=None, T0=None) -> np.ndarray:
    """K = hm T0 - hm (B/a) f(a) f(a)^T (real, symmetric, energy-independent)."""
    if mesh is None:
        mesh = lagrange_mesh(p.nlag, p.a)
    if T0 is None:
        T0 = kinetic_bloch(p.nlag, p.a, mesh)
    f_a = mesh["f_a"]
    return p.hm * T0 - p.hm * (p.bloch_B / p.a) * np.outer(f_a, f_a)


def point_coupling(p, V: np.ndarray, mesh) -> np.ndarray:
    """W[j, al, al'] = V_{al al'}(r_j) + delta_{al al'} (hm l(l+1)/r_j^2 + E_al - E)."""
    Vm = np.asarray(V).transpose(2, 1, 0)          # V[c2, c1, j] -> [j, c1, c2]
    W = np.array(Vm, dtype=np.complex128)
    d = channel_diagonal(p, mesh)                  # [al, j]
    for al in range(p.nch):
        W[:, al, al] += d[al]
    return W


def schur_matrix(p, V: np.ndarray, mesh=None, T0=None) -> np.ndarray:
    """S (N x N, radial-major): S[(i,al),(j,al')] = delta + Kinv[i,j] W[j, al, al']."""
    if mesh is None:
        mesh = lagrange_mesh(p.nlag, p.a)
    K = kinetic_matrix(p, mesh, T0)
    Kinv = np.linalg.inv(K)
    W = point_coupling(p, V, mesh)
    nch, nlag = p.nch, p.nlag
    S = np.zeros((nlag, nch, nlag, nch), dtype=np.complex128)
    for i in range(nlag):
        for j in range(nlag):
            S[i, :, j, :] = Kinv[i, j] * W[j]
        S[i, :, i, :] += np.eye(nch)
    return S.reshape(nlag * nch, nlag * nch)


def schur_rhs(p, mesh=None, T0=None) -> np.ndarray:
    """b~[(i,al), be] = sum_j Kinv[i,j] f_j(a) delta_{al be}  (N x nch, radial-major)."""
    if mesh is None:
        mesh = lagrange_mesh(p.nlag, p.a)
    Kinv = np.linalg.inv(kinetic_matrix(p, mesh, T0))
    g = Kinv @ mesh["f_a"]
    b = np.zeros((p.nlag, p.nch, p.nch), dtype=np.complex128)
    for al in range(p.nch):
        b[:, al, al] = g
    return b.reshape(p.nlag * p.nch, p.nch)


def radial_to_channel(p, Y: np.ndarray) -> np.ndarray:
    """Rows (i, al) -> (al, i)."""
    return np.ascontiguousarray(
        Y.reshape(p.nlag, p.nch, -1).transpose(1, 0, 2).reshape(p.nch * p.nlag, -1))


def channel_to_radial(p, X: np.ndarray) -> np.ndarray:
    """Rows (al, i) -> (i, al)."""
    return np.ascontiguousarray(
        X.reshape(p.nch, p.nlag, -1).transpose(1, 0, 2).reshape(p.nch * p.nlag, -1))


def woodbury_solve(p, V: np.ndarray, mesh=None, T0=None) -> np.ndarray:
    """X (channel-major, N x nch) from S x~ = b~ (oracle LU), reordered."""
    S = schur_matrix(p, V, mesh, T0)
    b = schur_rhs(p, mesh, T0)
    return radial_to_channel(p, solve(S, b))
