"""Exact / high-precision evaluations used to pin the oracle.

Nothing here shares arithmetic with ``oracle/``: the normalized associated
Legendre functions are built from their definition (Section 2.3, eq.
association, with P_l from the Rodrigues formula printed beside it) using
exact rational polynomial coefficients, and the prefactors are evaluated in
50-digit mpmath arithmetic.
"""

from fractions import Fraction
from functools import lru_cache
from math import comb, factorial

import pytest

# a host without mpmath skips the modules that import this one instead of
# failing their collection
mpmath = pytest.importorskip("mpmath")

mpmath.mp.dps = 50


@lru_cache(maxsize=None)
def legendre_poly_coeffs(k):
    """Exact coefficients c_0..c_k of P_k(x) = (1/(2^k k!)) d^k/dx^k (x^2-1)^k."""
    # (x^2 - 1)^k = sum_j C(k, j) (-1)^(k-j) x^(2j)
    poly = [Fraction(0)] * (2 * k + 1)
    for j in range(k + 1):
        poly[2 * j] = Fraction(comb(k, j) * (-1) ** (k - j))
    for _ in range(k):
        poly = [poly[i] * i for i in range(1, len(poly))]
    scale = Fraction(1, 2 ** k * factorial(k))
    return tuple(c * scale for c in poly)


@lru_cache(maxsize=None)
def dm_legendre_coeffs(m, k):
    """Exact coefficients of d^m/dx^m P_k(x)."""
    poly = list(legendre_poly_coeffs(k))
    for _ in range(m):
        poly = [poly[i] * i for i in range(1, len(poly))] or [Fraction(0)]
    return tuple(poly)


def pbar_exact(m, k, x):
    """P-bar^m_k(x) from eq. association, as an mpmath number (50 digits)."""
    x = mpmath.mpf(x)
    poly = dm_legendre_coeffs(m, k)
    val = mpmath.mpf(0)
    for c in reversed(poly):
        val = val * x + mpmath.mpf(c.numerator) / c.denominator
    pref = mpmath.sqrt(mpmath.mpf(2 * k + 1) / 2 * mpmath.factorial(k - m) / mpmath.factorial(k + m))
    return pref * (1 - x * x) ** (mpmath.mpf(m) / 2) * val
