"""Physics pins for the oracle's full pipeline (matrix, solve, R, U).

What the method fixes independently of any implementation:
  * zero potential -> U = 1 (zero phase shift), for any l and thresholds;
  * a square well filling (0, a): closed-form phase shift;
  * real potentials -> U unitary and symmetric; absorptive (W < 0) -> |U| < 1;
  * results independent of the channel radius a once V(a) ~ 0;
  * direct ODE integration of Eq. (cc_schrodinger) matched to the free
    asymptotics (single channel and coupled channels with thresholds).
Each pin also runs against planted mistakes in a copy of the oracle to show
that it would catch them.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import cc_problems as cp
import oracle
from oracle import collision as CL
from oracle import mesh as M
from oracle import system as S
from oracle.refine import truth_solve


def run(p, V=None, T0_fn=None, rnorm=1.0, drop_thresh=False):
    """Oracle pipeline with optional planted mistakes (used by the mutation tests)."""
    m = M.lagrange_mesh(p.nlag, p.a)
    T0 = (T0_fn or M.kinetic_bloch)(p.nlag, p.a, m)
    if V is None:
        V = cp.potential_at(p, m["r"])
    q = p
    if drop_thresh:
        import copy
        q = copy.copy(p)
        q.thresh = np.zeros_like(p.thresh)
    C, Phi = S.assemble_dense(q, V, m, T0)
    X, _ = truth_solve(C, Phi, steps=2)
    R = rnorm * CL.r_matrix(p, X, m["f_a"])
    U, nopen = CL.collision_matrix(p, R)
    return U, m


def zero_potential_problem(nch=4, nlag=50):
    p = cp.make_problem(3, nch, nlag, 10.0)
    p.thresh = np.array([0.0, 1.0, 2.0, 3.0])[:nch]
    p.s[:] = 0
    p.V0 = 0.0
    p.W = 0.0
    return p


def test_zero_potential_gives_identity():
    U, _ = run(zero_potential_problem())
    assert np.max(np.abs(U - np.eye(U.shape[0]))) < 1e-10


def square_well_U(V0, E=10.0, a=15.0, hm=cp.HM_1AMU):
    k = np.sqrt(E / hm)
    K = np.sqrt((E - V0) / hm + 0j)
    z = (k / K) * np.tan(K * a)
    # tan(ka + delta) = z  ->  U = e^{2 i delta} = e^{-2ika} (1 + iz) / (1 - iz)
    return np.exp(-2j * k * a) * (1 + 1j * z) / (1 - 1j * z)


@pytest.mark.parametrize("V0", [-50 - 10j, -50.0, 20.0, -3 - 0.5j])
def test_square_well_closed_form(V0):
    p = cp.make_problem(1, 1, 60, 10.0)
    V = np.full((1, 1, p.nlag), V0, dtype=np.complex128)
    U, _ = run(p, V=V)
    assert abs(U[0, 0] - square_well_U(V0)) < 1e-10


def test_real_potential_unitary_symmetric():
    p = cp.config1()
    p.W = 0.0
    U, _ = run(p)
    n = U.shape[0]
    assert np.max(np.abs(U.conj().T @ U - np.eye(n))) < 1e-12
    assert np.max(np.abs(U - U.T)) < 1e-12


def test_absorptive_potential_subunitary_symmetric():
    U, _ = run(cp.config1())
    assert np.max(np.linalg.eigvalsh(U.conj().T @ U)) < 1.0
    assert np.max(np.abs(U - U.T)) < 1e-12


def test_closed_channels_open_block_unitary():
    p = cp.config1()
    p.W = 0.0
    p.E = 3.0
    p.thresh = np.array([0.0, 1.0, 4.0, 4.5])
    U, _ = run(p)
    assert U.shape == (2, 2)
    assert np.max(np.abs(U.conj().T @ U - np.eye(2))) < 1e-12
    assert np.max(np.abs(U - U.T)) < 1e-12


@pytest.mark.parametrize("closed", [False, True])
def test_channel_radius_invariance(closed):
    p15 = cp.config1()
    if closed:
        p15.E = 3.0
        p15.thresh = np.array([0.0, 1.0, 4.0, 4.5])
    p18 = cp.make_problem(p15.seed, 4, 60, p15.E, a=18.0)
    p18.thresh, p18.s = p15.thresh.copy(), p15.s.copy()
    U15, _ = run(p15)
    U18, _ = run(p18)
    assert np.max(np.abs(U15 - U18)) < 2e-6          # WS tail at r = 15 fm is ~1e-7 of the depth


def _ode_regular_solutions(p, a):
    """Regular solutions of the coupled equations (Eq. cc_schrodinger), one per channel."""
    nch = p.nch
    l = np.asarray(p.l, dtype=float)

    def Vmat(r):
        return cp.potential_at(p, np.array([r]))[:, :, 0].T      # [c1, c2]

    def rhs(r, y):
        u = y[:nch * nch].reshape(nch, nch)
        du = y[nch * nch:].reshape(nch, nch)
        Wm = Vmat(r) / p.hm + np.diag(l * (l + 1) / r ** 2 + (np.asarray(p.thresh) - p.E) / p.hm)
        return np.concatenate([du.ravel(), (Wm @ u).ravel()])

    r0 = 1e-5
    u0 = np.diag(r0 ** (l + 1)).astype(np.complex128)
    du0 = np.diag((l + 1) * r0 ** l).astype(np.complex128)
    sol = solve_ivp(rhs, (r0, a), np.concatenate([u0.ravel(), du0.ravel()]),
                    method="DOP853", rtol=1e-12, atol=1e-30)
    y = sol.y[:, -1]
    return y[:nch * nch].reshape(nch, nch), y[nch * nch:].reshape(nch, nch)


def _ode_U(p):
    """U from matching Psi = k^-1/2 (I A - O U A) at r = a, without any R-matrix."""
    Psi, dPsi = _ode_regular_solutions(p, p.a)
    is_open, k, I, O, dI, dO = CL.channel_functions(p)
    assert np.all(is_open)
    P = np.sqrt(k)[:, None] * Psi
    Q = dPsi / np.sqrt(k)[:, None]
    A = (dO[:, None] * P - O[:, None] * Q) / (dO * I - O * dI)[:, None]
    D = (dI[:, None] * P - I[:, None] * Q) / (I * dO - dI * O)[:, None]
    return D @ np.linalg.inv(A)


def test_single_channel_woods_saxon_vs_ode():
    for l in (0, 2):
        p = cp.make_problem(5, 1, 60, 10.0)
        p.l = np.array([l], dtype=np.int32)
        U, _ = run(p)
        assert abs(U[0, 0] - _ode_U(p)[0, 0]) < 1e-8


def test_coupled_channels_with_thresholds_vs_ode():
    p = cp.make_problem(21, 3, 60, 10.0)          # l = 0,1,2; thresholds U(0,5); couplings U(-5,5)
    U, _ = run(p)
    Uo = _ode_U(p)
    assert np.max(np.abs(U - Uo)) < 1e-8


# ---- planted mistakes: each must be caught by at least one pin above ----------

def _T0_flip_offdiag(nlag, a, m):
    T = M.kinetic_bloch(nlag, a, m)
    return 2 * np.diag(np.diag(T)) - T


def test_mutation_kinetic_sign_is_caught():
    U, _ = run(zero_potential_problem(), T0_fn=_T0_flip_offdiag)
    assert np.max(np.abs(U - np.eye(U.shape[0]))) > 1e-3


def test_mutation_r_normalisation_is_caught():
    p = cp.make_problem(1, 1, 60, 10.0)
    V = np.full((1, 1, p.nlag), -50.0 + 0j)
    U, _ = run(p, V=V, rnorm=p.a)                      # forgot the 1/a
    assert abs(U[0, 0] - square_well_U(-50.0)) > 1e-3


def test_mutation_dropped_threshold_is_caught():
    p = cp.make_problem(21, 3, 60, 10.0)
    U, _ = run(p, drop_thresh=True)
    assert np.max(np.abs(U - _ode_U(p))) > 1e-3
