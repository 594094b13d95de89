"""Lagrange-Legendre mesh on (0, a) and the kinetic + Bloch matrix (oracle).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

The paper expands each channel's radial function in n Lagrange-Legendre basis
functions f_i(r) on the Gauss-Legendre mesh of (0, a), with the Lagrange
property f_i(r_j) = delta_ij / sqrt(lambda_j) (Sec. 2, theoretical
background), following Baye (Phys. Rep. 565 (2015) 1) and Descouvemont
(CPC 200 (2016) 199).  The paper prints neither the basis nor the kinetic
matrix; this module uses the standard regularised ("by x") basis

    f_i(r) = (-1)^(n+i) * (r / (a x_i)) * sqrt(a x_i (1 - x_i))
             * P_n(2r/a - 1) / (r - a x_i),          i = 1..n,

with x_i the zeros of the shifted Legendre polynomial P_n(2x - 1).

Pins (tests/test_oracle_mesh.py): nodes and weights against
numpy.polynomial.legendre.leggauss; the Lagrange property and the boundary
values f_i(a) against a direct evaluation of the basis functions; the kinetic
matrix against the exact integral  int_0^a f_i'(r) f_j'(r) dr  evaluated by a
2n-point Gauss rule (exact for this degree-(2n-2) polynomial integrand).
"""
from __future__ import annotations

import numpy as np


def gauss_legendre_unit(n: int):
    """Zeros x_i (ascending) of P_n(2x-1) on (0,1) and Gauss weights on (0,1).

    1. Newton iteration in double on t = cos(theta), theta from the usual
       initial guesses pi (k - 1/4)/(n + 1/2), with the three-term recurrence
       (j+1) P_{j+1} = (2j+1) t P_j - j P_{j-1} and
       P_n'(t) = n (t P_n - P_{n-1}) / (t^2 - 1).
    2. Three Newton steps with t and P_j(t) in double-double arithmetic, the
       derivative in double (quadratic convergence from a 1e-16 start).
    3. x = (1 + t)/2 and 1 - x = (1 - t)/2 formed in double-double and
       rounded once, so both come out correctly rounded, also near 0 and 1.
    Weights 2/((1 - t^2) P_n'(t)^2) on (-1,1) with 1 - t^2 = 4 x (1 - x),
    halved for (0,1).

    The kinetic matrix is exact only at the true zeros; 1-ulp changes of
    all nodes move the collision matrix by ~1e-10 at nlag = 50, hence the
    correctly rounded nodes.
    """
    from .ddarith import dd_add, dd_div_d, dd_mul, dd_mul_d, quick_two_sum, two_sum
    if n < 1:
        raise ValueError("n must be >= 1")
    k = np.arange(1, n + 1)
    theta = np.pi * (k - 0.25) / (n + 0.5)          # t descending

    def pair(t):
        p0 = np.ones_like(t)
        p1 = t.copy()
        for j in range(1, n):
            p0, p1 = p1, ((2 * j + 1) * t * p1 - j * p0) / (j + 1)
        return (p1, p0) if n > 1 else (t, np.ones_like(t))

    for _ in range(100):
        t = np.cos(theta)
        pn, pm = pair(t)
        dp = n * (t * pn - pm) / (t * t - 1.0)
        step = pn / (-np.sin(theta) * dp)             # d/dtheta P_n(cos theta) = -sin P_n'
        theta = theta - step
        if np.max(np.abs(step)) < 1e-16:
            break
    th, tl = np.cos(theta), np.zeros(n)
    for _ in range(3):
        # P_j(t) in double-double
        p0h, p0l = np.ones(n), np.zeros(n)
        p1h, p1l = th.copy(), tl.copy()
        for j in range(1, n):
            ah, al = dd_mul(th, tl, p1h, p1l)
            ah, al = dd_mul_d(ah, al, float(2 * j + 1))
            bh, bl = dd_mul_d(p0h, p0l, float(j))
            ch, cl = dd_add(ah, al, -bh, -bl)
            ch, cl = dd_div_d(ch, cl, float(j + 1))
            p0h, p0l, p1h, p1l = p1h, p1l, ch, cl
        pnh, pnl = (p1h, p1l) if n > 1 else (th, tl)
        pmh = p0h if n > 1 else np.ones(n)
        dp = n * (th * pnh - pmh) / (th * th - 1.0)
        sh, sl = dd_div_d(pnh, pnl, dp)
        th, tl = dd_add(th, tl, -sh, -sl)
    s, e = two_sum(np.ones(n), th)
    xh, _ = quick_two_sum(s, e + tl)
    s, e = two_sum(np.ones(n), -th)
    oh, _ = quick_two_sum(s, e - tl)
    x, omx = xh / 2.0, oh / 2.0
    pn, pm = pair(th)
    # P_n'(t) = n (t P_n - P_{n-1}) / (t^2 - 1) with 1 - t^2 = 4 x (1 - x)
    dp = n * (pm - th * pn) / (4.0 * x * omx)
    w = 2.0 / (4.0 * x * omx * dp * dp) / 2.0
    order = np.argsort(x)
    return x[order], omx[order], w[order]


def lagrange_mesh(nlag: int, a: float):
    """Mesh of the paper's Sec. 2 on (0, a).

    Returns dict with
      x       zeros of P_n(2x-1), ascending, on (0,1)
      lam     Gauss weights on (0,1) (the paper's lambda_i on (0,a) is a*lam)
      r       mesh radii a * x_i (fm)
      f_a     boundary values f_i(a) = (-1)^(n+i) / sqrt(a x_i (1 - x_i)),
              i 1-based: the q2(r_i) of the paper's Type-1 algorithm (Sec. 3.1)
    """
    x, omx, lam = gauss_legendre_unit(nlag)
    i1 = np.arange(1, nlag + 1)
    f_a = np.where((nlag + i1) % 2 == 0, 1.0, -1.0) / np.sqrt(a * x * omx)
    return {"x": x, "omx": omx, "lam": lam, "r": a * x, "f_a": f_a, "a": float(a), "n": nlag}


def kinetic_bloch(nlag: int, a: float, mesh=None) -> np.ndarray:
    """T0 = matrix of (-d^2/dr^2 + L(0)) in the regularised basis, in fm^-2.

    With the Bloch operator L(0) = delta(r - a) d/dr, integration by parts
    gives T0_ij = int_0^a f_i'(r) f_j'(r) dr (f_i(0) = 0), a symmetric matrix.
    Closed forms (Baye 2015, regularised shifted-Legendre mesh):
      T0_ii = [(4n^2+4n+3) x_i(1-x_i) - 6 x_i + 1] / [3 a^2 x_i^2 (1-x_i)^2]
      T0_ij = (-1)^(i+j) / [a^2 sqrt(x_i x_j (1-x_i)(1-x_j))]
              * [n^2 + n + 1 + (x_i + x_j - 2 x_i x_j)/(x_i - x_j)^2
                 - 1/(1-x_i) - 1/(1-x_j)],                      i != j.
    Multiply by hbar^2/2mu (MeV fm^2) to get MeV.  Every operation below is a
    single IEEE double operation evaluated left to right (no powers, no fused
    multiply-add), so the value is reproducible bit for bit; entries with
    i < j are evaluated and mirrored, so T0 is exactly symmetric.
    """
    m = mesh if mesh is not None else lagrange_mesh(nlag, a)
    x, omx = [float(v) for v in m["x"]], [float(v) for v in m["omx"]]
    n = nlag
    a = float(a)
    c_diag = float(4 * n * n + 4 * n + 3)
    c_off = float(n * n + n) + 1.0
    T = np.empty((n, n))
    for i in range(n):
        xi, oi = x[i], omx[i]
        num = c_diag * xi * oi - 6.0 * xi + 1.0
        den = 3.0 * a * a * (xi * xi) * (oi * oi)
        T[i, i] = num / den
        for j in range(i + 1, n):                    # i < j; mirrored, so T == T^T exactly
            xj, oj = x[j], omx[j]
            sgn = 1.0 if (i + j) % 2 == 0 else -1.0
            d = xi - xj
            pre = sgn / (a * a * np.sqrt(xi * xj * oi * oj))
            brk = c_off + (xi + xj - 2.0 * xi * xj) / (d * d) - 1.0 / oi - 1.0 / oj
            T[i, j] = pre * brk
            T[j, i] = T[i, j]
    return T
