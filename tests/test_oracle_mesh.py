"""Pins for the oracle's mesh, boundary values and kinetic+Bloch matrix (Sec. 2).

Nothing here re-types the oracle's formulas: nodes/weights are checked against
numpy's leggauss (and mpmath where present), the basis is evaluated directly
from its definition, and the kinetic matrix against the exact integral
int_0^a f_i' f_j' dr computed by an independent quadrature.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle.mesh import gauss_legendre_unit, kinetic_bloch, lagrange_mesh


@pytest.mark.parametrize("n", [1, 2, 7, 50, 100])
def test_nodes_and_weights_match_leggauss(n):
    x, omx, w = gauss_legendre_unit(n)
    t, wt = L.leggauss(n)
    np.testing.assert_allclose(x, (1 + t) / 2, rtol=0, atol=2e-16)
    # numpy's own endpoint weights are good to ~2e-12 (checked against mpmath below)
    np.testing.assert_allclose(w, wt / 2, rtol=5e-12)
    np.testing.assert_allclose(x + omx, 1.0, rtol=0, atol=2.3e-16)
    assert np.all(np.diff(x) > 0)


@pytest.mark.parametrize("n", [50, 100])
def test_nodes_correctly_rounded(n):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x, omx, w = gauss_legendre_unit(n)
    for i in range(n):
        t = mp.mpf(2) * mp.mpf(x[i]) - 1
        for _ in range(5):
            P, Pm = mp.legendre(n, t), mp.legendre(n - 1, t)
            t -= P / (n * (t * P - Pm) / (t * t - 1))
        assert float((1 + t) / 2) == x[i]
        assert float((1 - t) / 2) == omx[i]
        P, Pm = mp.legendre(n, t), mp.legendre(n - 1, t)
        dP = n * (t * P - Pm) / (t * t - 1)
        w_exact = 1 / ((1 - t * t) * dP * dP)
        assert abs(float((w[i] - w_exact) / w_exact)) < 1e-13


def _basis(n, a, x):
    """f_i(r) and f_i'(r) evaluated straight from the regularised-basis definition."""
    def P(s):
        c = np.zeros(n + 1); c[-1] = 1
        return L.legval(s, c)

    def dP(s):
        c = np.zeros(n + 1); c[-1] = 1
        return L.legval(s, L.legder(c))

    def f(i, r):                      # i 0-based
        xi = x[i]
        ci = (-1) ** (n + i + 1) * np.sqrt(a * xi * (1 - xi)) / (a * xi)
        return ci * r * P(2 * r / a - 1) / (r - a * xi)

    def fp(i, r):
        xi = x[i]
        ci = (-1) ** (n + i + 1) * np.sqrt(a * xi * (1 - xi)) / (a * xi)
        s = 2 * r / a - 1
        d = r - a * xi
        return ci * ((P(s) + r * 2 / a * dP(s)) * d - r * P(s)) / d ** 2

    def f_at_node(i):                 # 0/0 limit at r = r_i (l'Hopital)
        xi = x[i]
        ci = (-1) ** (n + i + 1) * np.sqrt(a * xi * (1 - xi)) / (a * xi)
        return ci * a * xi * (2 / a) * dP(2 * xi - 1)
    return f, fp, f_at_node


@pytest.mark.parametrize("n,a", [(8, 5.0), (30, 15.0)])
def test_lagrange_property_and_boundary_values(n, a):
    m = lagrange_mesh(n, a)
    f, _, f_node = _basis(n, a, m["x"])
    for i in range(n):
        for j in range(n):
            v = f_node(i) if i == j else f(i, m["r"][j])
            want = 1 / np.sqrt(a * m["lam"][j]) if i == j else 0.0
            assert abs(v - want) < 1e-11 * abs(1 / np.sqrt(a * m["lam"][i]))
        # boundary value of the basis function at r = a
        assert abs(f(i, a) - m["f_a"][i]) < 1e-12 * abs(m["f_a"][i])


@pytest.mark.parametrize("n,a", [(6, 3.0), (20, 15.0), (50, 15.0)])
def test_kinetic_equals_exact_integral(n, a):
    m = lagrange_mesh(n, a)
    T0 = kinetic_bloch(n, a, m)
    _, fp, _ = _basis(n, a, m["x"])
    tq, wq = L.leggauss(2 * n)          # exact for the degree 2n-2 integrand f_i' f_j'
    rq = a * (tq + 1) / 2
    D = np.array([fp(i, rq) for i in range(n)])
    Tint = (D * (wq * a / 2)) @ D.T
    assert np.max(np.abs(T0 - Tint)) < 1e-10 * np.max(np.abs(Tint))
    assert np.array_equal(T0, T0.T)


def test_kinetic_zero_mode_structure():
    """sum_j T0_ij * r_j is the matrix of -d^2/dr^2 + L(0) on f = r, i.e. the
    Bloch term alone: int f_i' * 1 dr = f_i(a).  Exact for polynomials in the
    span of the basis (r is in it), so this pins T0's action independently."""
    n, a = 25, 10.0
    m = lagrange_mesh(n, a)
    T0 = kinetic_bloch(n, a, m)
    # coefficients of g(r) = r in the basis: c_j = g(r_j) sqrt(a lam_j)
    c = m["r"] * np.sqrt(a * m["lam"])
    lhs = T0 @ c
    assert np.max(np.abs(lhs - m["f_a"])) < 1e-10 * np.max(np.abs(m["f_a"]))
