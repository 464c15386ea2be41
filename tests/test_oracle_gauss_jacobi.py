"""Pins of the oracle's Gauss-Jacobi form (oracle/gauss_jacobi.py: Section 4,
Lemma distinct_theorem, Lemma quadratures, eqs. weights1, weights2,
weights2_0, transform, transform2).

None of these re-derives the oracle's own arithmetic:
  - at m = 0 and parity 0 the nodes and weights are the Gauss-Legendre
    rule of degree 2n (positive half, weights doubled): numpy's leggauss at
    small n, a 40-digit Newton solution (tests/_exact.py) at n = 60, 300;
  - both rules integrate (1 - x^2)^m x^{2k} exactly (the beta integral
    B(k + 1/2, m + 1) in closed form), the odd rule with sigma_n at x = 0;
  - at small sizes the nodes are zeros, and the weights the printed formula,
    of P-bar^m_N evaluated in 50-digit arithmetic from the exact Rodrigues
    polynomial (tests/_exact.py), with the derivative a central difference
    of those exact values;
  - the matrix of eqs. transform / transform2 is orthogonal, and its
    inverse map undoes the forward map;
  - planted mistakes (a dropped factor 1 - x^2, the even rule's degree for
    the odd parity, a shifted node) fail these pins.
"""

import math
from decimal import Decimal, localcontext

import numpy as np
import pytest

import oracle.gauss_jacobi as GJ
from tests import _exact


def beta_integral(k, m):
    """int_{-1}^{1} (1 - x^2)^m x^{2k} dx = B(k + 1/2, m + 1)."""
    return math.exp(math.lgamma(k + 0.5) + math.lgamma(m + 1) - math.lgamma(k + m + 1.5))


def rule_errors(m, p, n, x, w, sigma_n=None):
    """Relative errors of the rule on (1 - x^2)^m x^{2k} for every k it
    integrates exactly (Lemma quadratures: 2k <= 4n - 2, resp. 4n)."""
    errs = []
    for k in range(0, 2 * n + p):
        q = np.sum(w * np.exp(m * np.log1p(-x * x)) * x ** (2 * k))
        if p == 1 and k == 0:
            q += sigma_n
        errs.append(abs(q - beta_integral(k, m)) / beta_integral(k, m))
    return max(errs)


@pytest.mark.parametrize("n", [1, 7, 20])
def test_m0_even_is_gauss_legendre(n):
    """numpy's leggauss (its weights are accurate to ~1e-14 x degree only)."""
    x, w = GJ.gj_nodes_weights(0, 0, n)
    xg, wg = np.polynomial.legendre.leggauss(2 * n)
    assert np.max(np.abs(x - xg[n:])) < 4e-16
    assert np.max(np.abs(w - 2 * wg[n:]) / (2 * wg[n:])) < 2e-14 * 2 * n


@pytest.mark.parametrize("n", [60, 300])
def test_m0_even_is_gauss_legendre_extended_precision(n):
    """The Gauss-Legendre rule of degree 2n solved in 40-digit arithmetic
    (tests/_exact.py): rho_j = 2 w_j at m = 0."""
    x, w = GJ.gj_nodes_weights(0, 0, n)
    for j in range(0, n, max(1, n // 12)):
        xr, wr = _exact.gl_root_and_weight(2 * n, float(x[j]))
        assert abs(float(xr) - x[j]) <= 8 * np.spacing(x[j])
        assert abs(2 * float(wr) - w[j]) <= 1e-13 * w[j]


@pytest.mark.parametrize("m", [0, 3, 40, 200])
@pytest.mark.parametrize("p", [0, 1])
def test_rules_are_exact(m, p):
    n = 30
    x, w = GJ.gj_nodes_weights(m, p, n)
    assert x.shape == (n,) and np.all(np.diff(x) > 0) and 0 < x[0] and x[-1] < 1 and np.all(w > 0)
    sig = GJ.gj_sigma_n(m, n) if p == 1 else None
    assert rule_errors(m, p, n, x, w, sig) < 1e-11


def _exact_derivative(m, N, x):
    """d/dx P-bar^m_N at the float x: central difference of exact values
    with h = 1e-20 (error ~1e-40 relative)."""
    with localcontext() as c:
        c.prec = _exact.DIGITS
        h = Decimal("1e-20")
        xd = _exact.dec(x)
        return (_exact.pbar_exact(m, N, xd + h) - _exact.pbar_exact(m, N, xd - h)) / (2 * h)


@pytest.mark.parametrize("m,p,n", [(0, 0, 4), (2, 0, 3), (2, 1, 3), (5, 1, 2)])
def test_zeros_and_weights_in_exact_arithmetic(m, p, n):
    N = m + 2 * n + p
    x, w = GJ.gj_nodes_weights(m, p, n)
    for xi, wi in zip(x, w):
        d = _exact_derivative(m, N, float(xi))
        # a float within a few ulp of the zero: |P(x)| <= |P'| * 4 ulp(x)
        assert abs(_exact.pbar_exact(m, N, float(xi))) <= abs(d) * Decimal(4 * np.spacing(xi))
        with localcontext() as c:
            c.prec = _exact.DIGITS
            xd = _exact.dec(float(xi))
            w_exact = 2 * (2 * N + 1) / ((1 - xd * xd) * d * d)
        assert abs(float(w_exact) - wi) <= 1e-13 * wi


@pytest.mark.parametrize("m,p,n", [(0, 0, 50), (0, 1, 50), (60, 0, 60), (60, 1, 60), (400, 1, 100)])
def test_matrix_is_orthogonal(m, p, n):
    A = GJ.gj_matrix(m, p, n)
    assert np.max(np.abs(A.T @ A - np.eye(n))) < 1e-12
    assert np.max(np.abs(A @ A.T - np.eye(n))) < 1e-12


def test_inverse_undoes_forward_and_rows_agree():
    rng = np.random.default_rng(5)
    n, m = 80, 80
    for p in (0, 1):
        b = rng.uniform(-1, 1, (n, 2))
        a = GJ.gj_forward(b, m, p)
        assert np.max(np.abs(GJ.gj_inverse(a, m, p) - b)) < 1e-13
        rows = [0, 17, n - 1]
        assert np.max(np.abs(GJ.gj_forward(b, m, p, rows=rows) - a[rows])) < 1e-15


# ---- planted mistakes: each must fail one of the pins above


def test_planted_dropped_factor_fails_exactness():
    m, p, n = 3, 0, 30
    x, w = GJ.gj_nodes_weights(m, p, n)
    wrong = w * (1.0 - x * x)  # weights1 without its factor 1 / (1 - x^2)
    assert rule_errors(m, p, n, x, wrong) > 1e-3


def test_planted_even_degree_for_odd_parity_fails_exactness():
    m, n = 3, 30
    x, w = GJ.gj_nodes_weights(m, 0, n)  # zeros of P-bar^m_{m+2n} used as the odd rule
    assert rule_errors(m, 1, n, x, w, GJ.gj_sigma_n(m, n)) > 1e-3


def test_planted_shifted_node_fails_exact_zero():
    m, p, n = 2, 1, 3
    x, _ = GJ.gj_nodes_weights(m, p, n)
    xi = float(x[1]) * (1 + 1e-12)
    d = _exact_derivative(m, m + 2 * n + p, xi)
    assert abs(_exact.pbar_exact(m, m + 2 * n + p, xi)) > abs(d) * Decimal(4 * np.spacing(xi))
