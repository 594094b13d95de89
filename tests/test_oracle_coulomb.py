"""Pins for the charged-channel asymptotics (Coulomb and Whittaker functions).

Independent checks: mpmath's own Coulomb and Whittaker functions (arbitrary
precision, hypergeometric series; W'/W too, at Sommerfeld parameters up to the
42 of a closed alpha + 208Pb channel 1.5 MeV below threshold), the Wronskian F'G - FG' = 1, the eta -> 0
limits (pinned to scipy in test_oracle_special), and scattering physics:
a pure Coulomb interior matched to Coulomb functions has no nuclear phase
shift (U = 1), and a Woods-Saxon plus Coulomb system agrees with direct ODE
integration matched to mpmath's functions, closed channels included.
Planted mistakes in the Sommerfeld parameter are caught.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import cc_problems as cp
from oracle import collision as CL
from oracle import mesh as M
from oracle import system as S
from oracle.coulomb import coulomb_fg, turning_point, whittaker_logd, whittaker_w
from oracle.refine import truth_solve

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30


def _mp_coulomb(l, eta, rho):
    F = mp.coulombf(l, eta, rho)
    G = mp.coulombg(l, eta, rho)
    dF = mp.diff(lambda x: mp.coulombf(l, eta, x), rho)
    dG = mp.diff(lambda x: mp.coulombg(l, eta, x), rho)
    return float(F), float(G), float(dF), float(dG)


def _mp_whittaker(l, eta, rho):
    W = mp.whitw(-eta, l + 0.5, 2 * rho)
    dW = mp.diff(lambda x: mp.whitw(-eta, l + 0.5, 2 * x), rho)
    return float(W), float(dW)


# rho on both sides of the turning point; eta < 0 is an attractive pair
@pytest.mark.parametrize("l", [0, 1, 3, 8, 20])
@pytest.mark.parametrize("eta", [-4.0, 0.35, 2.5, 9.3, 16.2])
@pytest.mark.parametrize("rho", [0.7, 4.0, 13.0, 21.9, 38.0])
def test_coulomb_fg_vs_mpmath(l, eta, rho):
    got = coulomb_fg(l, eta, rho)
    ref = _mp_coulomb(l, eta, rho)
    for g, r in zip(got, ref):
        assert abs(g - r) <= 1e-10 * abs(r), (got, ref)
    F, G, dF, dG = got
    assert abs(dF * G - F * dG - 1.0) < 1e-11


@pytest.mark.parametrize("l,eta", [(0, 16.2), (4, 9.3), (20, 3.0)])
def test_coulomb_continuous_across_turning_point(l, eta):
    # the inner side comes from the inward integration, the outer from Steed's method
    tp = turning_point(l, eta)
    d = 1e-7 * tp
    F0, G0, dF0, dG0 = coulomb_fg(l, eta, tp - d)
    F1, G1, dF1, dG1 = coulomb_fg(l, eta, tp + d)
    assert abs(F1 - F0 - 2 * d * 0.5 * (dF0 + dF1)) <= 1e-11 * abs(F1)
    assert abs(G1 - G0 - 2 * d * 0.5 * (dG0 + dG1)) <= 1e-11 * abs(G1)
    # u'' = (l(l+1)/rho^2 + 2 eta/rho - 1) u vanishes at the turning point
    assert abs(dF1 - dF0) <= 1e-11 * abs(dF1)
    assert abs(dG1 - dG0) <= 1e-11 * abs(dG1)


@pytest.mark.parametrize("l", [0, 1, 2, 5])
@pytest.mark.parametrize("rho", [0.5, 3.0, 12.0])
def test_eta_zero_limits(l, rho):
    for a, b in zip(coulomb_fg(l, 0.0, rho), CL.riccati_bessel(l, rho)):
        assert abs(a - b) <= 1e-12 * abs(b)
    for a, b in zip(whittaker_w(l, 0.0, rho), CL.whittaker_reduced(l, rho)):
        assert abs(a - b) <= 1e-11 * abs(b)


@pytest.mark.parametrize("l", [0, 1, 4, 9])
@pytest.mark.parametrize("eta", [0.5, 4.0, 12.0])
@pytest.mark.parametrize("rho", [0.3, 2.0, 8.0, 25.0])
def test_whittaker_vs_mpmath(l, eta, rho):
    W, dW = whittaker_w(l, eta, rho)
    We, dWe = _mp_whittaker(l, eta, rho)
    assert abs(W - We) <= 1e-10 * abs(We)
    assert abs(dW - dWe) <= 1e-10 * abs(dWe)


@pytest.mark.parametrize("l", [0, 1, 5, 20])
@pytest.mark.parametrize("eta", [0.5, 12.0, 41.8])
@pytest.mark.parametrize("rho", [0.3, 2.0, 8.5, 30.0])
def test_whittaker_log_derivative_vs_mpmath(l, eta, rho):
    y = whittaker_logd(l, eta, rho)
    W, dW = _mp_whittaker(l, eta, rho)
    assert abs(y - dW / W) <= 1e-11 * abs(dW / W)


# ---- scattering physics ---------------------------------------------------

def run(p, V=None):
    m = M.lagrange_mesh(p.nlag, p.a)
    T0 = M.kinetic_bloch(p.nlag, p.a, m)
    if V is None:
        V = cp.potential_at(p, m["r"])
    C, Phi = S.assemble_dense(p, V, m, T0)
    X, _ = truth_solve(C, Phi, steps=2)
    R = CL.r_matrix(p, X, m["f_a"])
    return CL.collision_matrix(p, R)[0]


def pure_coulomb_problem(E, nch=3, closed=True):
    """Point-charge Coulomb interior, no nuclear potential, no couplings."""
    p = cp.charged_problem(7, nch, 100, E, V0=0.0, W=0.0, Rc=0.0)
    p.s[:] = 0.0
    p.l = np.array([0, 2, 3][:nch], dtype=np.int32)
    p.thresh = np.array([0.0, 1.5, E + 4.0][:nch]) if closed else np.zeros(nch)
    return p


@pytest.mark.parametrize("E", [10.0, 30.0])   # below / above the barrier (about 20 MeV)
def test_pure_coulomb_interior_gives_identity(E):
    U = run(pure_coulomb_problem(E))
    assert U.shape == (2, 2)
    assert np.max(np.abs(U - np.eye(2))) < 1e-8


def _ode_U_charged(p):
    """U from direct integration of the coupled equations, matched at r = a to
    mpmath's Coulomb (open) and Whittaker (closed) functions, no R-matrix."""
    nch = p.nch
    l = np.asarray(p.l, dtype=float)
    ecm = p.E - np.asarray(p.thresh)
    k = np.sqrt(np.abs(ecm) / p.hm)
    eta = np.asarray(p.zz) / (2.0 * p.hm * k)

    def rhs(r, y):
        u = y[:nch * nch].reshape(nch, nch)
        du = y[nch * nch:].reshape(nch, nch)
        V = cp.potential_at(p, np.array([r]))[:, :, 0].T
        Wm = V / p.hm + np.diag(l * (l + 1) / r ** 2 - ecm / p.hm)
        return np.concatenate([du.ravel(), (Wm @ u).ravel()])

    # regular solutions ~ (r/r0)^(l+1), started at unit size so that the
    # absolute tolerance stays far below them whatever l is
    r0 = 1e-4
    y0 = np.concatenate([np.eye(nch, dtype=complex).ravel(),
                         np.diag((l + 1) / r0).astype(complex).ravel()])
    sol = solve_ivp(rhs, (r0, p.a), y0, method="DOP853", rtol=1e-12, atol=1e-30)
    Psi = sol.y[:nch * nch, -1].reshape(nch, nch)
    dPsi = sol.y[nch * nch:, -1].reshape(nch, nch)
    I = np.zeros(nch, complex); O = np.zeros(nch, complex)
    dI = np.zeros(nch, complex); dO = np.zeros(nch, complex)
    for c in range(nch):
        rho = k[c] * p.a
        if ecm[c] > 0:
            F, G, dF, dG = _mp_coulomb(int(l[c]), eta[c], rho)
            I[c], O[c], dI[c], dO[c] = G - 1j * F, G + 1j * F, dG - 1j * dF, dG + 1j * dF
        else:
            O[c], dO[c] = _mp_whittaker(int(l[c]), eta[c], rho)
    # u(a) = Psi alpha = k^-1/2 (e_c0 I - diag(O) x);  du/dr = k^1/2 (e_c0 I' - diag(O') x)
    op = np.flatnonzero(ecm > 0)
    U = np.zeros((op.size, op.size), complex)
    sk = np.sqrt(k)
    for j, c0 in enumerate(op):
        A = np.zeros((2 * nch, 2 * nch), complex)
        b = np.zeros(2 * nch, complex)
        A[:nch, :nch] = Psi
        A[:nch, nch:] = np.diag(O / sk)
        A[nch:, :nch] = dPsi
        A[nch:, nch:] = np.diag(dO * sk)
        b[c0] = I[c0] / sk[c0]
        b[nch + c0] = dI[c0] * sk[c0]
        x = np.linalg.solve(A, b)[nch:]
        U[:, j] = x[op]
    return U


# Point-charge Coulomb (Rc = 0) in the ODE pins: the kink of the uniform-sphere
# potential at Rc slows the mesh convergence of the Gauss quadrature to ~1e-6.
def test_charged_coupled_channels_with_closed_channel_vs_ode():
    p = cp.charged_problem(21, 3, 120, 30.0, Rc=0.0)
    p.thresh = np.array([0.0, 4.0, 33.0])        # channel 2 closed
    U = run(p)
    Uo = _ode_U_charged(p)
    assert U.shape == (2, 2)
    assert np.max(np.abs(U - Uo)) < 1e-8


def test_single_channel_grazing_vs_ode():
    """One channel at l = 20 near the grazing energy of the alpha + 208Pb case."""
    p = cp.charged_problem(5, 1, 120, 25.0, Rc=0.0)
    p.l = np.array([20], dtype=np.int32)
    U = run(p)
    Uo = _ode_U_charged(p)
    assert abs(U[0, 0] - Uo[0, 0]) < 1e-8
    assert 0.0 < abs(U[0, 0]) < 1.0               # absorptive


# ---- planted mistakes -----------------------------------------------------

def test_mutation_eta_sign_is_caught(monkeypatch):
    orig = CL.sommerfeld
    monkeypatch.setattr(CL, "sommerfeld", lambda p, k: -orig(p, k))
    U = run(pure_coulomb_problem(30.0, closed=False))
    assert np.max(np.abs(U - np.eye(U.shape[0]))) > 1e-3


def test_mutation_eta_factor_two_is_caught(monkeypatch):
    orig = CL.sommerfeld
    monkeypatch.setattr(CL, "sommerfeld", lambda p, k: 2.0 * orig(p, k))
    U = run(pure_coulomb_problem(30.0, closed=False))
    assert np.max(np.abs(U - np.eye(U.shape[0]))) > 1e-3
