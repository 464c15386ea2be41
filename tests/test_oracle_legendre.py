"""Pins for oracle.legendre: closed forms, the definition, identities and
library routines that share no arithmetic with the oracle's recurrence."""

import math
from decimal import Decimal

import numpy as np
import pytest
from scipy import special

import oracle
from tests._exact import diagonal_exact, pbar_exact

try:  # a library routine used as one pin; the test fails (not skips) without it
    import mpmath
except ImportError:  # pragma: no cover
    mpmath = None

XS = np.array([-0.97, -0.61, -0.2, 0.0, 0.13, 0.5, 0.77, 0.999])


def test_closed_forms():
    """Section 2.3, eq. association: P-bar^0_0 = 1/sqrt 2, P-bar^0_1 = sqrt(3/2) x,
    P-bar^1_1 = (sqrt 3 / 2) sqrt(1-x^2), P-bar^0_2 = sqrt(5/2) (3x^2 - 1)/2."""
    x = XS
    t0 = oracle.legendre_table(0, x, 2)
    np.testing.assert_allclose(t0[0], 1 / math.sqrt(2), rtol=1e-15)
    np.testing.assert_allclose(t0[1], math.sqrt(1.5) * x, rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(t0[2], math.sqrt(2.5) * (3 * x * x - 1) / 2, rtol=1e-14)
    t1 = oracle.legendre_table(1, x, 1)
    np.testing.assert_allclose(t1[0], math.sqrt(3) / 2 * np.sqrt((1 - x) * (1 + x)), rtol=1e-15)


@pytest.mark.parametrize("k", range(0, 16))
def test_matches_definition_exactly_for_low_degrees(k):
    """eq. association with P_l from the Rodrigues formula, in exact rational
    polynomials + 50-digit prefactors, for every m <= k <= 15."""
    for m in range(k + 1):
        got = oracle.legendre_table(m, XS, k)[-1]
        ref = np.array([float(pbar_exact(m, k, xv)) for xv in XS])
        # roundoff of the degree recurrence: about k ulp of max P-bar (<= 1.3 here)
        np.testing.assert_allclose(got, ref, rtol=2e-14, atol=1e-14)


@pytest.mark.parametrize("k,m", [(40, 0), (40, 17), (300, 3), (700, 100), (1999, 3)])
def test_high_degree_against_mpmath(k, m):
    """Library routine (mpmath Ferrers function, arbitrary precision) with the
    Condon-Shortley sign removed and the eq. association normalization, at
    points where its hypergeometric evaluation converges quickly."""
    assert mpmath is not None, "this pin needs mpmath (pip package 'mpmath')"
    mpmath.mp.dps = 40
    pts = np.array([-0.8, -0.3, 0.3, 0.6, 0.9])
    got = oracle.legendre_table(m, pts, k)[-1]
    for xv, g in zip(pts, got):
        norm = mpmath.sqrt(mpmath.mpf(2 * k + 1) / 2 * mpmath.factorial(k - m) / mpmath.factorial(k + m))
        ref = float((-1) ** m * norm * mpmath.legenp(k, m, mpmath.mpf(xv), type=2))
        assert abs(g - ref) <= 1e-12 * max(abs(ref), 1.0), (k, m, xv, g, ref)


@pytest.mark.parametrize("m", [10, 500, 1500, 2047])
def test_diagonal_closed_form_through_underflow(m):
    """eq. association at l = m: d^m/dx^m P_m = (2m)!/(2^m m!), so
    P-bar^m_m(x) = sqrt((2m+1)/2) sqrt((2m)!)/(2^m m!) (1-x^2)^{m/2}, evaluated
    in 50-digit decimal arithmetic at the l = 1024 Gauss-Legendre nodes.  Values below
    the float64 range must come out (near) zero; representable ones to
    (m + 10) * 4e-16 relative, which exercises the exponent tracking of Section 4."""
    x, _ = oracle.gl_nodes_weights(2048)
    pts = x[::37]
    got = oracle.legendre_table(m, pts, m)[0]
    for xv, g in zip(pts, got):
        ref = diagonal_exact(m, float(xv))
        if ref > Decimal("1e-290"):
            # sqrt(1-x^2) carries ~1 ulp, amplified m times by the m-th power
            assert abs(g - float(ref)) <= 4e-16 * (m + 10) * float(ref), (m, xv, g, ref)
        else:
            assert abs(g) < 1e-280


@pytest.mark.parametrize("m", [1000, 1500, 2000, 2046])
def test_large_order_columns_orthonormal_at_l1024(m):
    """The columns P-bar^m_{m+p+2j} start far below the float64 range near the
    poles and grow through it; GL orthonormality (Section 2.3 + eq. thetas)
    only holds if the tracked exponents are right everywhere."""
    for p in (0, 1):
        import oracle.sht as osht
        A = osht.unit_matrix(1024, m, p)
        if A.shape[1]:
            np.testing.assert_allclose(A.T @ A, np.eye(A.shape[1]), atol=1e-13)


@pytest.mark.parametrize("k", [5, 6, 64, 300, 1023])
def test_unsold_sum(k):
    """Addition theorem at coincident points (Unsold): sum_{m=-k}^{k}
    P-bar_k^{|m|}(x)^2 = (2k+1)/2 for the orthonormal functions of eq.
    association."""
    s = np.zeros_like(XS)
    for m in range(k + 1):
        v = oracle.legendre_table(m, XS, k)[-1]
        s += (1.0 if m == 0 else 2.0) * v * v
    np.testing.assert_allclose(s, (2 * k + 1) / 2, rtol=1e-13)


@pytest.mark.parametrize("k", [10, 200, 700])
def test_addition_theorem(k):
    """sum_{m=-k}^{k} P-bar_k^{|m|}(x1) P-bar_k^{|m|}(x2) e^{i m (phi1-phi2)}
    = (2k+1)/2 P_k(cos gamma), cos gamma = x1 x2 + s1 s2 cos(phi1-phi2),
    with P_k from scipy (library routine)."""
    rng = np.random.default_rng(11)
    x1 = rng.uniform(-0.95, 0.95, size=3)
    x2 = rng.uniform(-0.95, 0.95, size=3)
    dphi = rng.uniform(0, 2 * np.pi, size=3)
    pts = np.concatenate([x1, x2])
    tab = np.array([oracle.legendre_table(m, pts, k)[-1] for m in range(k + 1)])  # (k+1, 6)
    t1, t2 = tab[:, :3], tab[:, 3:]
    ms = np.arange(k + 1)[:, None]
    wgt = np.where(ms == 0, 1.0, 2.0)
    lhs = np.sum(wgt * t1 * t2 * np.cos(ms * dphi[None, :]), axis=0)
    cg = x1 * x2 + np.sqrt(1 - x1 * x1) * np.sqrt(1 - x2 * x2) * np.cos(dphi)
    rhs = (2 * k + 1) / 2 * special.eval_legendre(k, cg)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * (2 * k + 1)), (k, lhs, rhs)


@pytest.mark.parametrize("m", [0, 1, 3, 100, 900])
def test_paper_x2_recurrence_holds(m):
    """Section 2.3, eqs. c_rec, d_rec, recurrence0 and recurrence (the x^2
    three-term recurrence that the product uses): x^2 P-bar_l = c_{l-2}
    P-bar_{l-2} + d_l P-bar_l + c_l P-bar_{l+2}.  The oracle evaluates with the
    x recurrence, so this pins its values against the paper's constants."""

    def c(l):
        return math.sqrt((l - m + 1) * (l - m + 2) * (l + m + 1) * (l + m + 2)
                         / ((2 * l + 1) * (2 * l + 3) ** 2 * (2 * l + 5)))

    def d(l):
        return (2 * l * (l + 1) - 2 * m * m - 1) / ((2 * l - 1) * (2 * l + 3))

    x = np.array([-0.9, -0.3, 0.05, 0.4, 0.8, 0.95])
    kmax = m + 300
    T = oracle.legendre_table(m, x, kmax)
    for l in range(m, kmax - 1):
        i = l - m
        lhs = x * x * T[i]
        terms = [d(l) * T[i], c(l) * T[i + 2]]
        if l >= m + 2:
            terms.append(c(l - 2) * T[i - 2])
        rhs = sum(terms)
        scale = np.abs(lhs) + sum(np.abs(t) for t in terms) + 1e-300
        assert np.all(np.abs(lhs - rhs) <= 1e-13 * scale), (m, l)


def test_against_scipy_lpmv_small_degree():
    """scipy's unnormalized associated Legendre function (library routine),
    with its Condon-Shortley sign removed and eq. association's normalization."""
    for k in range(0, 25):
        for m in range(0, k + 1):
            norm = math.sqrt((2 * k + 1) / 2 * math.factorial(k - m) / math.factorial(k + m))
            ref = (-1) ** m * norm * special.lpmv(m, k, XS)
            got = oracle.legendre_table(m, XS, k)[-1]
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)


def test_orthonormal_on_interval():
    """Section 2.3: for fixed m the P-bar^m_k are orthonormal on (-1, 1).
    Integrated with numpy's own Gauss-Legendre rule (library routine; 64
    points are exact for the degree <= 120 products used here)."""
    xq, wq = np.polynomial.legendre.leggauss(64)
    for m in [0, 1, 2, 5, 30]:
        T = oracle.legendre_table(m, xq, m + 30)
        gram = (T * wq) @ T.T
        np.testing.assert_allclose(gram, np.eye(T.shape[0]), atol=1e-13)


def test_parity():
    """Section 2.3: P-bar^m_l(-x) = (-1)^{l-m} P-bar^m_l(x)."""
    x = np.abs(XS[XS != 0])
    for m in [0, 2, 7, 50]:
        a = oracle.legendre_table(m, x, m + 40)
        b = oracle.legendre_table(m, -x, m + 40)
        sign = (-1.0) ** np.arange(a.shape[0])
        np.testing.assert_allclose(b, sign[:, None] * a, rtol=1e-14, atol=1e-300)
