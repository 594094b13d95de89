"""Pins for the Woodbury-kinetic (Type 3) form of the system in the oracle.

What fixes S independently of the formula that builds it: multiplying it back by
I_nch (x) K must give the matrix M that oracle.system assembles from Eq.
(block_structure) on its own; its reordered solution must equal the direct
solution of M X = Phi; K and so K^-1 do not depend on the energy, so S(E2) - S(E1)
is -(E2 - E1) Kinv (x) I; and a planted index mistake fails the first pin.
"""
import numpy as np
import pytest

import cc_problems as cp
from oracle import mesh as M
from oracle import system as S
from oracle import woodbury as WB
from oracle.refine import truth_solve


def setup(p):
    m = M.lagrange_mesh(p.nlag, p.a)
    T0 = M.kinetic_bloch(p.nlag, p.a, m)
    V = cp.potential_at(p, m["r"])
    return m, T0, V


@pytest.mark.parametrize("B", [0.0, -1.3])
def test_kinetic_times_schur_gives_back_the_matrix(B):
    p = cp.make_problem(41, 3, 12, 7.0)
    p.bloch_B = B
    m, T0, V = setup(p)
    C, _ = S.assemble_dense(p, V, m, T0)
    Smat = WB.schur_matrix(p, V, m, T0)
    K = WB.kinetic_matrix(p, m, T0)
    KS = np.kron(K, np.eye(p.nch)) @ Smat             # radial-major I (x) K is K (x) I_nch
    back = WB.radial_to_channel(p, WB.radial_to_channel(p, KS).T).T
    assert np.max(np.abs(back - C)) < 1e-10 * np.max(np.abs(C))


def test_schur_solution_equals_direct_solution():
    p = cp.config1()
    m, T0, V = setup(p)
    C, Phi = S.assemble_dense(p, V, m, T0)
    X_direct, _ = truth_solve(C, Phi, steps=2)
    X_wb = WB.woodbury_solve(p, V, m, T0)
    assert np.max(np.abs(X_wb - X_direct)) < 1e-10 * np.max(np.abs(X_direct))


def test_schur_rhs_is_kinv_of_surface_vectors():
    p = cp.make_problem(43, 4, 20, 5.0)
    m, T0, _ = setup(p)
    b = WB.radial_to_channel(p, WB.schur_rhs(p, m, T0))
    Phi = S.surface_rhs(p, m)
    K = WB.kinetic_matrix(p, m, T0)
    back = np.kron(np.eye(p.nch), K) @ b                  # channel-major I (x) K
    assert np.max(np.abs(back - Phi)) < 1e-11 * np.max(np.abs(Phi))


def test_kinetic_inverse_is_energy_independent():
    p1 = cp.make_problem(44, 3, 15, 6.0)
    p2 = cp.make_problem(44, 3, 15, 9.5)
    m, T0, V = setup(p1)
    S1 = WB.schur_matrix(p1, V, m, T0)
    S2 = WB.schur_matrix(p2, V, m, T0)
    Kinv = np.linalg.inv(WB.kinetic_matrix(p1, m, T0))
    expect = -(p2.E - p1.E) * np.kron(Kinv, np.eye(p1.nch))
    assert np.max(np.abs((S2 - S1) - expect)) < 1e-10 * np.max(np.abs(expect))


def test_mutation_coupling_at_wrong_point_is_caught(monkeypatch):
    p = cp.make_problem(41, 3, 12, 7.0)
    m, T0, V = setup(p)
    C, _ = S.assemble_dense(p, V, m, T0)
    orig = WB.point_coupling
    # V_{al al'} taken at the reversed mesh order: r_i in place of r_j for i != j
    monkeypatch.setattr(WB, "point_coupling", lambda p, V, mesh: orig(p, V, mesh)[::-1])
    Smat = WB.schur_matrix(p, V, m, T0)
    K = WB.kinetic_matrix(p, m, T0)
    back = WB.radial_to_channel(p, WB.radial_to_channel(p, np.kron(K, np.eye(p.nch)) @ Smat).T).T
    assert np.max(np.abs(back - C)) > 1e-3 * np.max(np.abs(C))
