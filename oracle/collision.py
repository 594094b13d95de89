"""R-matrix contraction and collision matrix U (oracle).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

R-matrix (Sec. 3.1 step 4): R_{al be} = sum_i q2(r_i) X[(al,i), be], with
q2(r_i) = f_i(a).  The paper leaves the normalisation implicit; with C in MeV
(hbar^2/2mu = hm explicit) the dimensionless R-matrix is

    R = (hm / a) * Phi^T X,        X = C^{-1} Phi,

so that u(a) = R (a u'(a) - B u(a)) channel by channel.

Collision matrix (the "matching to the asymptotic solutions at a" of Sec. 1;
Coulomb/Whittaker functions of Sec. 4.1).  For eta = 0 the open-channel
functions are Riccati-Bessel: F_l(rho) = rho j_l(rho), G_l(rho) = -rho y_l(rho),
I = G - iF, O = G + iF, rho = k a, k = sqrt((E - E_c)/hm).  With
u_c(r) = k_c^{-1/2} [delta_{c c0} I_c(k_c r) - U_{c c0} O_c(k_c r)] and
R~ = a sqrt(k) R sqrt(k):

    U = (diag O - R~ diag O')^{-1} (diag I - R~ diag I'),   O' = dO/drho,

restricted to open x open.  A closed channel (E < E_c) uses k = sqrt((E_c - E)/hm),
O = reduced Whittaker W~_l(rho) = e^{-rho} sum_{k=0}^{l} (l+k)!/(k!(l-k)!) (2 rho)^{-k}
(= sqrt(2 rho / pi) K_{l+1/2}(rho)) and I = 0.  A Bloch constant B replaces
O' -> O' - (B/rho) O and I' -> I' - (B/rho) I.

Pins (tests/test_oracle_special.py, test_oracle_physics.py): F, G against
scipy.special.spherical_jn / spherical_yn, the Wronskian F'G - FG' = 1,
W~ against scipy.special.kv; physics invariants (zero potential -> U = 1,
square-well closed form, unitarity/symmetry for real V, channel-radius
invariance, ODE integration, |U| < 1 with absorption).
"""
from __future__ import annotations

import math

import numpy as np

from .lu import solve


def r_matrix(p, X: np.ndarray, f_a: np.ndarray) -> np.ndarray:
    """R[al, be] = (hm / a) sum_i f_i(a) X[(al, i), be]."""
    X3 = X.reshape(p.nch, p.nlag, -1)
    return (p.hm / p.a) * np.einsum("i,aib->ab", f_a, X3)


def _double_factorial_odd(m: int) -> float:
    """(2m+1)!! = 1*3*5*...*(2m+1)."""
    out = 1.0
    for q in range(1, 2 * m + 2, 2):
        out *= q
    return out


def riccati_bessel(l: int, rho: float):
    """Return (F_l, G_l, F_l', G_l') at rho > 0 (derivatives w.r.t. rho).

    G by upward recurrence from G_0 = cos, G_1 = cos/rho + sin (stable).
    F by upward recurrence from F_0 = sin, F_1 = sin/rho - cos when rho >= l + 1,
    else by its power series rho^(l+1) sum_k (-rho^2/2)^k / (k! (2l+2k+1)!!).
    Derivatives: X_l' = X_{l-1} - (l/rho) X_l  (X_0' = cos for F, -sin for G).
    """
    if rho <= 0:
        raise ValueError("rho must be positive")
    s, c = math.sin(rho), math.cos(rho)

    def up(x0, x1, L):
        xs = [x0, x1]
        for q in range(1, L):
            xs.append((2 * q + 1) / rho * xs[q] - xs[q - 1])
        return xs

    G = up(c, c / rho + s, max(l, 1))

    def f_series(L):
        term = rho ** (L + 1) / _double_factorial_odd(L)
        acc = term
        k = 0
        while True:
            k += 1
            term *= -(rho * rho / 2.0) / (k * (2 * L + 2 * k + 1))
            acc += term
            if abs(term) < 1e-18 * abs(acc):
                return acc

    if rho >= l + 1:
        F = up(s, s / rho - c, max(l, 1))
    else:
        F = [f_series(L) for L in range(max(l, 1) + 1)]
    if l == 0:
        return F[0], G[0], c, -s
    Fl, Gl = F[l], G[l]
    dF = F[l - 1] - l / rho * Fl
    dG = G[l - 1] - l / rho * Gl
    return Fl, Gl, dF, dG


def whittaker_reduced(l: int, rho: float):
    """Return (W~_l(rho), dW~_l/drho) for eta = 0 (decaying closed-channel solution)."""
    w = 0.0
    dw = 0.0
    for k in range(l + 1):
        ck = math.factorial(l + k) / (math.factorial(k) * math.factorial(l - k))
        t = ck * (2.0 * rho) ** (-k)
        w += t
        dw += t * (-1.0 - k / rho)
    e = math.exp(-rho)
    return e * w, e * dw


def sommerfeld(p, k: np.ndarray) -> np.ndarray:
    """eta_c = zz_c / (2 hm k_c) (zz = Z1 Z2 e^2 of the channel; 0 when neutral)."""
    zz = getattr(p, "zz", None)
    if zz is None:
        return np.zeros_like(k)
    return np.asarray(zz, dtype=np.float64) / (2.0 * p.hm * k)


def channel_functions(p):
    """Per-channel (open, k, I, O, I', O') at rho = k a (Bloch-shifted derivatives).

    Neutral channels (eta = 0) take the Riccati-Bessel and reduced Whittaker
    functions below; charged ones the Coulomb functions F_l(eta, rho),
    G_l(eta, rho) and the Whittaker function W_{-eta,l+1/2}(2 rho) of
    oracle.coulomb, with the same I = G - iF, O = G + iF (open) and I = 0 for
    closed channels, where O = 1, O' = W'/W (a closed channel's column of the
    matching matrix scales with O, so U depends on W'/W only).
    """
    from .coulomb import coulomb_fg, whittaker_logd

    ecm = p.E - np.asarray(p.thresh, dtype=np.float64)
    if np.any(ecm == 0.0):
        raise ValueError("a channel sits exactly at threshold")
    is_open = ecm > 0
    k = np.sqrt(np.abs(ecm) / p.hm)
    eta = sommerfeld(p, k)
    I = np.zeros(p.nch, dtype=np.complex128)
    O = np.zeros(p.nch, dtype=np.complex128)
    dI = np.zeros(p.nch, dtype=np.complex128)
    dO = np.zeros(p.nch, dtype=np.complex128)
    for c in range(p.nch):
        rho = k[c] * p.a
        if is_open[c]:
            if eta[c] == 0.0:
                F, G, dF, dG = riccati_bessel(int(p.l[c]), rho)
            else:
                F, G, dF, dG = coulomb_fg(int(p.l[c]), float(eta[c]), rho)
            I[c], O[c] = G - 1j * F, G + 1j * F
            dI[c], dO[c] = dG - 1j * dF, dG + 1j * dF
        else:
            if eta[c] == 0.0:
                w, dw = whittaker_reduced(int(p.l[c]), rho)
            else:   # only W'/W enters U: O = 1, O' = W'/W
                w, dw = 1.0, whittaker_logd(int(p.l[c]), float(eta[c]), rho)
            O[c], dO[c] = w, dw
        dI[c] -= p.bloch_B / rho * I[c]
        dO[c] -= p.bloch_B / rho * O[c]
    return is_open, k, I, O, dI, dO


def collision_matrix(p, R: np.ndarray):
    """Return (U, nopen): U is nopen x nopen complex128, open channels in index order."""
    is_open, k, I, O, dI, dO = channel_functions(p)
    sk = np.sqrt(k)
    Rt = p.a * sk[:, None] * R * sk[None, :]
    ZO = np.diag(O) - Rt * dO[None, :]
    ZI = np.diag(I) - Rt * dI[None, :]
    idx = np.flatnonzero(is_open)
    if idx.size == 0:
        return np.zeros((0, 0), dtype=np.complex128), 0
    Ufull = solve(ZO, ZI[:, idx])
    return Ufull[idx, :], int(idx.size)
