"""Exact / high-precision evaluations used to pin the oracle.

Nothing here shares arithmetic with ``oracle/``: the normalized associated
Legendre functions are built from their definition (Section 2.3, eq.
association, with P_l from the Rodrigues formula printed beside it) using
exact rational polynomial coefficients, and the square roots of the
prefactors are taken in 50-digit decimal arithmetic.  Only the standard
library is used (``fractions``, ``decimal``), so these pins run on every host:
a missing optional package can never turn them into skips.
"""

from decimal import Decimal, localcontext
from fractions import Fraction
from functools import lru_cache
from math import comb, factorial

DIGITS = 50


def dec(q):
    """A Fraction, int or float as a Decimal rounded to DIGITS digits (floats
    are converted exactly first)."""
    if isinstance(q, float):
        q = Fraction(q)
    q = Fraction(q)
    with localcontext() as c:
        c.prec = DIGITS
        return Decimal(q.numerator) / Decimal(q.denominator)


def dsqrt(q):
    """sqrt of a non-negative rational, to DIGITS digits."""
    with localcontext() as c:
        c.prec = DIGITS + 5
        r = dec(q).sqrt()
    with localcontext() as c:
        c.prec = DIGITS
        return +r


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
    """P-bar^m_k(x) from eq. association as a Decimal (DIGITS digits): the
    polynomial d^m P_k / dx^m and (1 - x^2)^{floor(m/2)} exactly in rationals
    (x, a float, converted exactly), the remaining square roots rounded."""
    xq = Fraction(x)
    val = Fraction(0)
    for c in reversed(dm_legendre_coeffs(m, k)):
        val = val * xq + c
    r = 1 - xq * xq
    rational = val * r ** (m // 2)
    pref2 = Fraction(2 * k + 1, 2) * Fraction(factorial(k - m), factorial(k + m))
    with localcontext() as c:
        c.prec = DIGITS
        out = dec(rational) * dsqrt(pref2)
        if m % 2:
            out = out * dsqrt(r)
        return +out


def diagonal_exact(m, x):
    """P-bar^m_m(x) = sqrt((2m+1)/2) sqrt((2m)!)/(2^m m!) (1-x^2)^{m/2} (eq.
    association at degree m, where d^m P_m/dx^m = (2m)!/(2^m m!)), as a
    Decimal; the power is taken in DIGITS + 10 digit arithmetic."""
    c2 = Fraction(2 * m + 1, 2) * Fraction(factorial(2 * m), (2 ** m * factorial(m)) ** 2)
    r = 1 - Fraction(x) ** 2
    with localcontext() as c:
        c.prec = DIGITS + 10
        c.Emin = -10 ** 8
        p = dec(r) ** (m // 2)
        if m % 2:
            p = p * dsqrt(r)
        out = dsqrt(c2) * p
    with localcontext() as c:
        c.prec = DIGITS
        c.Emin = -10 ** 8
        return +out


def gl_root_and_weight(n, x0, digits=40, steps=5):
    """The zero of P_n nearest to the float x0 and its Gauss-Legendre weight
    w = 2 / ((1 - x^2) P_n'(x)^2) (Section 2, eq. thetas), by Newton's method
    on the integer-coefficient recurrence (j + 1) P_{j+1} = (2j + 1) x P_j -
    j P_{j-1} in `digits`-digit decimal arithmetic.  Returns Decimals."""
    with localcontext() as c:
        c.prec = digits

        def pp(x):
            p0, p1 = Decimal(1), x
            for j in range(1, n):
                p0, p1 = p1, ((2 * j + 1) * x * p1 - j * p0) / (j + 1)
            return p1, p0

        x = Decimal(x0)
        for _ in range(steps):
            a, b = pp(x)
            x = x - a / (n * (x * a - b) / (x * x - 1))
        a, b = pp(x)
        dp = n * (x * a - b) / (x * x - 1)
        return +x, 2 / ((1 - x * x) * dp * dp)
