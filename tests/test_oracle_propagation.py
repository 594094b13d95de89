"""Pins for the R-matrix propagation of the oracle (sectors beyond the first).

Independent checks: the sector basis built as explicit numpy polynomials
(Lagrange property, boundary values, the exact integral of f_i' f_j'); a sector
with no potential must carry the exact log-derivative of the regular free
solution (Riccati-Bessel F_l) from one end to the other; U with 2 or 3 sectors
must equal U from one sector over the same (0, a), neutral and charged; a
planted sign mistake in the propagation formula is caught.
"""
import numpy as np
import numpy.polynomial.polynomial as npp
import pytest

import cc_problems as cp
from oracle import collision as CL
from oracle import propagation as P
from oracle.pipeline import oracle_solve


def _explicit_basis(n, r1, r2):
    """f_i as numpy polynomials in x = (r - r1)/h (coefficients), from the nodes."""
    sm = P.sector_mesh(n, r1, r2)
    h = r2 - r1
    x, lam = (sm["r"] - r1) / h, sm["lam"]
    polys = []
    for i in range(n):
        c = npp.polyfromroots(np.delete(x, i))
        polys.append(c / npp.polyval(x[i], c) / np.sqrt(lam[i]))
    return sm, x, h, polys


# monomial coefficients lose digits to cancellation as n grows (at n = 12 the
# explicit K is no longer symmetric to 1e-3): small n here, the free-sector pin
# below covers n = 30
@pytest.mark.parametrize("n,r1,r2", [(6, 2.0, 5.0), (8, 4.0, 15.0)])
def test_sector_basis_against_explicit_polynomials(n, r1, r2):
    tol = 1e-9 if n <= 6 else 1e-7
    sm, x, h, polys = _explicit_basis(n, r1, r2)
    for i, c in enumerate(polys):
        vals = npp.polyval(x, c)
        expect = np.zeros(n)
        expect[i] = 1.0 / np.sqrt(sm["lam"][i])
        assert np.allclose(vals, expect, atol=tol * np.max(np.abs(expect)))
        assert abs(npp.polyval(0.0, c) - sm["fL"][i]) <= tol * max(1.0, abs(sm["fL"][i]))
        assert abs(npp.polyval(1.0, c) - sm["fR"][i]) <= tol * max(1.0, abs(sm["fR"][i]))
    # int_{r1}^{r2} f_i' f_j' dr = (1/h) int_0^1 (d f_i/dx)(d f_j/dx) dx
    K = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            integ = npp.polyint(npp.polymul(npp.polyder(polys[i]), npp.polyder(polys[j])))
            K[i, j] = (npp.polyval(1.0, integ) - npp.polyval(0.0, integ)) / h
    assert np.max(np.abs(K - sm["Kf"])) < 10 * tol * np.max(np.abs(K))


@pytest.mark.parametrize("l", [0, 2])
@pytest.mark.parametrize("r1,r2", [(5.0, 9.0), (3.0, 12.0)])
def test_free_sector_carries_riccati_log_derivative(l, r1, r2):
    E = 10.0
    q = cp.make_problem(1, 1, 30, E)
    q.l = np.array([l], dtype=np.int32)
    k = np.sqrt(E / q.hm)
    sm = P.sector_mesh(30, r1, r2)
    g = P.sector_green(q, np.zeros((1, 1, 30), complex), sm)

    def Rl(r):
        F, _, dF, _ = CL.riccati_bessel(l, k * r)
        return F / (k * dF)                    # u / u' of the regular solution F_l(kr)
    out = P.propagate(np.array([[Rl(r1)]]), g)[0, 0]
    assert abs(out - Rl(r2)) < 1e-9 * max(1.0, abs(Rl(r2)))


@pytest.mark.parametrize("radii,nlag", [([0, 7.5, 15], 40), ([0, 5, 10, 15], 30), ([0, 9, 15], 40)])
def test_sectors_reproduce_single_sector(radii, nlag):
    p1 = cp.make_problem(21, 3, 60, 10.0)
    ref = oracle_solve(p1, refine_steps=2)
    q = cp.make_problem(21, 3, nlag, 10.0)
    U, R, nopen = P.propagated_collision(q, radii, lambda r: cp.potential_at(q, r))
    assert nopen == ref["nopen"]
    assert np.max(np.abs(U - ref["U"])) < 1e-9


def test_charged_sectors_reproduce_single_sector():
    p1 = cp.charged_problem(22, 2, 120, 30.0, Rc=0.0)
    ref = oracle_solve(p1, refine_steps=2)
    q = cp.charged_problem(22, 2, 60, 30.0, Rc=0.0)
    U, _, _ = P.propagated_collision(q, [0, 8.0, 16.0], lambda r: cp.potential_at(q, r))
    assert np.max(np.abs(U - ref["U"])) < 1e-8


def test_mutation_propagation_sign_is_caught(monkeypatch):
    def bad(Rl, g):
        gLL, gLR, gRL, gRR = g
        return gRR - gRL @ np.linalg.solve(Rl - gLL, gLR)
    monkeypatch.setattr(P, "propagate", bad)
    p1 = cp.make_problem(21, 3, 60, 10.0)
    ref = oracle_solve(p1, refine_steps=2)
    q = cp.make_problem(21, 3, 40, 10.0)
    U, _, _ = P.propagated_collision(q, [0, 7.5, 15], lambda r: cp.potential_at(q, r))
    assert np.max(np.abs(U - ref["U"])) > 1e-3
