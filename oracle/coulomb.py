"""Coulomb and Whittaker functions for charged channels (oracle).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

Sec. 4.1 lists, among the asymptotic functions the collision matrix is built
from, the Coulomb functions of Barnett's COULFG (Steed's method) and the
Whittaker functions of closed channels.  For a channel of Sommerfeld
parameter eta = Z1 Z2 e^2 / (2 hm k) the open-channel functions are the
regular and irregular Coulomb functions F_l(eta, rho), G_l(eta, rho) of the
Coulomb equation

    u''(rho) = (l(l+1)/rho^2 + 2 eta/rho - 1) u(rho),

normalised by the Wronskian F'G - FG' = 1, and a closed channel (E < E_c,
k = sqrt((E_c - E)/hm), eta = Z1 Z2 e^2 / (2 hm k)) uses the decaying solution of

    u''(rho) = (l(l+1)/rho^2 + 2 eta/rho + 1) u(rho),

the Whittaker function W_{-eta, l+1/2}(2 rho).

Steed's method, in the notation S_L = L/rho + eta/L, R_L = sqrt(1 + eta^2/L^2),
T_L = S_L + S_{L+1}:

  CF1:  f = F_l'/F_l = S_{l+1} - R_{l+1}^2/(T_{l+1} - R_{l+2}^2/(T_{l+2} - ...)),
        which is the backward recurrence g_L = R_L^2/(T_L - g_{L+1}) with
        g_L = R_L F_L/F_{L-1} (from the ladder relations of F in L), so that
        f = S_{l+1} - g_{l+1} and sign F_l = prod_L sign g_L once the start
        L lies beyond the turning point (where F_L > 0);
  CF2:  p + iq = (G' + iF')/(G + iF)
             = i(1 - eta/rho) + (i/rho) a_1/(b_1 + a_2/(b_2 + ...)),
        a_k = (i eta + l + k)(i eta - l + k - 1),  b_k = 2(rho - eta + k i);
  then with gamma = (f - p)/q the Wronskian gives
        F = sign / sqrt(q (1 + gamma^2)),  F' = f F,  G = gamma F,
        G' = (p gamma - q) F.

Both continued fractions are evaluated here backwards from a finite depth
that is doubled until the value stops changing, the plainest evaluation of a
continued fraction.  Inside the Coulomb turning point rho_tp = eta +
sqrt(eta^2 + l(l+1)) q is exponentially small next to p and CF2 loses its
accuracy; there G, G' are taken from Steed's method at rho_tp and carried
inward by integrating the Coulomb equation (G grows inward, so inward
integration is stable), and F = 1/(f G - G') follows from the Wronskian.
The Whittaker function is started from its asymptotic expansion

    W_{-eta, l+1/2}(2 rho) ~ e^{-rho} (2 rho)^{-eta}
                             sum_k (l+1+eta)_k (eta-l)_k / k! (-1/(2 rho))^k

at a radius where the terms fall below double precision, and integrated
inward the same way (the decaying solution also grows inward).  The collision
matrix needs only W'/W (a closed channel's column of the matching matrix scales
with W), which whittaker_logd integrates as a Riccati equation: that stays
finite where W itself over- or underflows (large eta, small rho).

The integrations use scipy's DOP853 at rtol 1e-13.  Pins
(tests/test_oracle_coulomb.py): F, G, F', G' and W, W' against mpmath's
independent implementations, the Wronskian, the eta -> 0 limits (Riccati-
Bessel functions and the reduced Whittaker function of this oracle), and the
physics pins of charged-channel scattering (a pure Coulomb interior gives
U = 1; Woods-Saxon plus Coulomb against ODE integration matched to mpmath's
Coulomb functions).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def turning_point(l: int, eta: float) -> float:
    """Outer classical turning point of the Coulomb equation at unit energy."""
    return eta + math.sqrt(eta * eta + l * (l + 1.0))


def _cf1_depth(l: int, eta: float, rho: float, M: int):
    """f = F_l'/F_l and sign(F_l) from the CF1 truncated at L = l + M."""
    g = 0.0
    sign = 1
    for L in range(l + M, l, -1):
        S_L = L / rho + eta / L
        S_L1 = (L + 1) / rho + eta / (L + 1)
        g = (1.0 + (eta / L) ** 2) / (S_L + S_L1 - g)
        if g < 0:
            sign = -sign
    f = (l + 1) / rho + eta / (l + 1) - g
    return f, sign


def coulomb_cf1(l: int, eta: float, rho: float):
    """CF1 of Steed's method: (f = F_l'/F_l, sign of F_l) at rho > 0."""
    # start beyond the turning point of the top L so that F_{l+M} > 0
    M = 16
    while (l + M) * (l + M + 1.0) <= rho * rho - 2.0 * eta * rho:
        M *= 2
    f_old, _ = _cf1_depth(l, eta, rho, M)
    for _ in range(40):
        M *= 2
        f, sign = _cf1_depth(l, eta, rho, M)
        if abs(f - f_old) <= 1e-15 * abs(f):
            return f, sign
        f_old = f
    raise ArithmeticError(f"CF1 did not converge (l={l}, eta={eta}, rho={rho})")


def _cf2_depth(l: int, eta: float, rho: float, M: int) -> complex:
    t = 0j
    for k in range(M, 0, -1):
        a_k = (1j * eta + l + k) * (1j * eta - l + k - 1)
        b_k = 2.0 * (rho - eta + 1j * k)
        t = a_k / (b_k + t)
    return 1j * (1.0 - eta / rho) + (1j / rho) * t


def coulomb_cf2(l: int, eta: float, rho: float) -> complex:
    """CF2 of Steed's method: p + iq = (G' + iF')/(G + iF) at rho > 0."""
    M = 16
    v_old = _cf2_depth(l, eta, rho, M)
    for _ in range(24):
        M *= 2
        v = _cf2_depth(l, eta, rho, M)
        if abs(v - v_old) <= 1e-15 * abs(v):
            return v
        v_old = v
    raise ArithmeticError(f"CF2 did not converge (l={l}, eta={eta}, rho={rho})")


def _steed(l: int, eta: float, rho: float):
    f, sign = coulomb_cf1(l, eta, rho)
    pq = coulomb_cf2(l, eta, rho)
    p, q = pq.real, pq.imag
    gamma = (f - p) / q
    F = sign / math.sqrt(q * (1.0 + gamma * gamma))
    return F, gamma * F, f * F, (p * gamma - q) * F


def _integrate(l: int, eta: float, sgn: float, r0: float, u0: float, du0: float, r1: float):
    """Carry (u, u') of u'' = (l(l+1)/r^2 + 2 eta/r + sgn) u from r0 to r1."""
    ll = l * (l + 1.0)

    def rhs(r, y):
        return [y[1], (ll / (r * r) + 2.0 * eta / r + sgn) * y[0]]

    sol = solve_ivp(rhs, (r0, r1), [u0, du0], method="DOP853", rtol=1e-13, atol=0.0)
    if not sol.success:
        raise ArithmeticError(sol.message)
    return float(sol.y[0, -1]), float(sol.y[1, -1])


def coulomb_fg(l: int, eta: float, rho: float):
    """(F_l, G_l, F_l', G_l') of the Coulomb functions at rho > 0 (derivatives in rho)."""
    if rho <= 0:
        raise ValueError("rho must be positive")
    tp = turning_point(l, eta)
    if rho >= tp:
        return _steed(l, eta, rho)
    _, G_tp, _, dG_tp = _steed(l, eta, tp)
    G, dG = _integrate(l, eta, -1.0, tp, G_tp, dG_tp, rho)
    f, _ = coulomb_cf1(l, eta, rho)
    F = 1.0 / (f * G - dG)
    return F, G, f * F, dG


def whittaker_logd(l: int, eta: float, rho: float) -> float:
    """W'/W (rho-derivative) of W_{-eta, l+1/2}(2 rho), for any eta >= 0.

    y = u'/u of the decaying solution obeys the Riccati equation y' = Q - y^2,
    Q = 1 + 2 eta/rho + l(l+1)/rho^2, and is stable when integrated inward
    (a deviation from the decaying branch y ~ -sqrt(Q) shrinks like
    exp(-2 int sqrt(Q))).  It is started from the WKB value -sqrt(Q) - Q'/(4Q)
    at rho + 40, where that start's error has decayed by more than e^-80 on
    arrival, so no normalisation (and no overflow of W itself) is involved.
    """
    if rho <= 0:
        raise ValueError("rho must be positive")
    ll = l * (l + 1.0)

    def Q(r):
        return 1.0 + 2.0 * eta / r + ll / (r * r)

    rb = rho + 40.0
    dQ = -2.0 * eta / (rb * rb) - 2.0 * ll / rb ** 3
    y0 = -math.sqrt(Q(rb)) - dQ / (4.0 * Q(rb))
    sol = solve_ivp(lambda r, y: [Q(r) - y[0] * y[0]], (rb, rho), [y0], method="DOP853",
                    rtol=1e-13, atol=1e-14)
    if not sol.success:
        raise ArithmeticError(sol.message)
    return float(sol.y[0, -1])


def whittaker_w(l: int, eta: float, rho: float):
    """(W, dW/drho) of W_{-eta, l+1/2}(2 rho), the decaying closed-channel function."""
    if rho <= 0:
        raise ValueError("rho must be positive")
    rb = max(rho, 2.0 * abs(eta) + l + 20.0)
    for _ in range(30):
        # asymptotic series at rb; accept when its smallest term is negligible
        s, ds = 1.0, -1.0 - eta / rb     # sum t_k and sum t_k (-1 - (eta+k)/rb)
        t = 1.0
        ok = False
        for k in range(1, 2000):
            t_new = t * (l + k + eta) * (eta - l + k - 1) / k * (-1.0 / (2.0 * rb))
            if abs(t_new) > abs(t) and k > 1:
                break
            t = t_new
            s += t
            ds += t * (-1.0 - (eta + k) / rb)
            if abs(t) < 1e-17 * abs(s):
                ok = True
                break
        if ok:
            break
        rb *= 2.0
    else:
        raise ArithmeticError("Whittaker asymptotic series did not converge")
    # W = e^{-rb} (2 rb)^{-eta} s and, term by term,
    # dW/drho = e^{-rb} (2 rb)^{-eta} sum_k t_k (-1 - (eta + k)/rb) = e^{-rb} (2 rb)^{-eta} ds
    lnw = -rb - eta * math.log(2.0 * rb)
    w0, dw0 = s, ds
    if rb == rho:
        e = math.exp(lnw)
        return e * w0, e * dw0
    w, dw = _integrate(l, eta, +1.0, rb, w0, dw0, rho)
    e = math.exp(lnw)
    return e * w, e * dw
