"""Double-double error-free transformations for the oracle's "truth" residual.

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench's CPU legs.

The paper computes the refinement residual r = b - M x in double precision
(Sec. 3.2, Sec. 3.4 step 7).  To measure the FP64 GPU path against something
more accurate than itself, the oracle evaluates that residual in double-double
arithmetic:

  two_sum(a, b)  -> (s, e) with s = fl(a + b), a + b = s + e exactly (Knuth);
  two_prod(a, b) -> (p, e) with p = fl(a * b), a * b = p + e exactly
                    (Dekker's splitting with the constant 2^27 + 1; valid
                    while |a|,|b| < 2^995, far above any value here).

Pins (tests/test_oracle_dd.py): exactness against Python's Fraction on random
and adversarial doubles, and the dd residual against an exact rational
residual on a small system.
"""
from __future__ import annotations

import numpy as np

_SPLIT = 134217729.0  # 2^27 + 1


def two_sum(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    lo = a - hi
    return hi, lo


def two_prod(a, b):
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def quick_two_sum(a, b):
    """Normalise (a, b) with |a| >= |b|: s = fl(a + b), e = exact remainder."""
    s = a + b
    e = b - (s - a)
    return s, e


def dd_add(xh, xl, yh, yl):
    """(xh + xl) + (yh + yl) in double-double (sloppy add, ~2^-104 relative)."""
    s, e = two_sum(xh, yh)
    e = e + (xl + yl)
    return two_sum(s, e)


def dd_mul(xh, xl, yh, yl):
    """(xh + xl) * (yh + yl) in double-double."""
    p, e = two_prod(xh, yh)
    e = e + (xh * yl + xl * yh)
    return quick_two_sum(p, e)


def dd_mul_d(xh, xl, b):
    """(xh + xl) * b for a double b, in double-double."""
    p, e = two_prod(xh, b)
    e = e + xl * b
    return quick_two_sum(p, e)


def dd_div_d(xh, xl, b):
    """(xh + xl) / b for a double b, in double-double."""
    q1 = xh / b
    p, e = two_prod(q1, b)
    r = ((xh - p) - e + xl) / b
    return quick_two_sum(q1, r)


def dd_accumulate_products(a: np.ndarray, b: np.ndarray):
    """sum_k a[..., k] * b[..., k] of real float64 arrays, in double-double.

    Returns (hi, lo) with hi + lo the sum to ~2^-104 relative of its terms.
    """
    p, pe = two_prod(a, b)
    hi = np.zeros(p.shape[:-1])
    lo = np.zeros(p.shape[:-1])
    for k in range(p.shape[-1]):
        hi, lo = dd_add(hi, lo, p[..., k], pe[..., k])
    return hi, lo


def dd_residual(C: np.ndarray, X: np.ndarray, B: np.ndarray) -> np.ndarray:
    """r = B - C X for complex matrices, accumulated in double-double.

    Real and imaginary parts are expanded into real products:
      Re(CX) = sum_k Cr Xr - Ci Xi,   Im(CX) = sum_k Cr Xi + Ci Xr,
    each term accumulated exactly-rounded to double-double, then B added and
    the result rounded to complex128.
    """
    n, m = C.shape[0], X.shape[1]
    Cr, Ci = C.real, C.imag
    Xr, Xi = X.real, X.imag
    out = np.empty((n, m), dtype=np.complex128)
    for col in range(m):
        xr = Xr[:, col][None, :]
        xi = Xi[:, col][None, :]
        # stack the four real product sequences along the summation axis
        ar = np.concatenate([Cr, -Ci], axis=1)
        br = np.concatenate([np.broadcast_to(xr, Cr.shape), np.broadcast_to(xi, Ci.shape)], axis=1)
        ai = np.concatenate([Cr, Ci], axis=1)
        bi = np.concatenate([np.broadcast_to(xi, Cr.shape), np.broadcast_to(xr, Ci.shape)], axis=1)
        hr, lr = dd_accumulate_products(ar, br)
        hi_, li = dd_accumulate_products(ai, bi)
        # B - (h + l)
        rr_h, rr_l = dd_add(B[:, col].real, np.zeros(n), -hr, -lr)
        ri_h, ri_l = dd_add(B[:, col].imag, np.zeros(n), -hi_, -li)
        out[:, col] = (rr_h + rr_l) + 1j * (ri_h + ri_l)
    return out
