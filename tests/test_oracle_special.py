"""Pins for the asymptotic functions (eta = 0): scipy special functions + Wronskian."""
import numpy as np
import pytest
import scipy.special as sp

from oracle.collision import riccati_bessel, whittaker_reduced


@pytest.mark.parametrize("l", [0, 1, 2, 3, 5])
@pytest.mark.parametrize("rho", [0.05, 0.3, 1.0, 2.9, 6.0, 10.3, 23.7])
def test_riccati_bessel_vs_scipy(l, rho):
    F, G, dF, dG = riccati_bessel(l, rho)
    j, y = sp.spherical_jn(l, rho), sp.spherical_yn(l, rho)
    jp, yp = sp.spherical_jn(l, rho, derivative=True), sp.spherical_yn(l, rho, derivative=True)
    Fe, Ge = rho * j, -rho * y
    dFe, dGe = j + rho * jp, -(y + rho * yp)
    assert abs(F - Fe) <= 1e-12 * abs(Fe) + 1e-300
    assert abs(G - Ge) <= 1e-12 * abs(Ge)
    assert abs(dF - dFe) <= 1e-11 * abs(dFe) + 1e-300
    assert abs(dG - dGe) <= 1e-12 * abs(dGe)
    assert abs(dF * G - F * dG - 1.0) < 1e-12          # Wronskian


@pytest.mark.parametrize("l", [0, 1, 2, 3, 6])
@pytest.mark.parametrize("rho", [0.2, 1.0, 4.0, 15.0])
def test_whittaker_vs_scipy_kv(l, rho):
    W, dW = whittaker_reduced(l, rho)
    We = np.sqrt(2 * rho / np.pi) * sp.kv(l + 0.5, rho)
    h = 1e-5 * rho
    dWe = (np.sqrt(2 * (rho + h) / np.pi) * sp.kv(l + 0.5, rho + h)
           - np.sqrt(2 * (rho - h) / np.pi) * sp.kv(l + 0.5, rho - h)) / (2 * h)
    assert abs(W - We) < 1e-13 * abs(We)
    assert abs(dW - dWe) < 1e-8 * abs(dWe)
