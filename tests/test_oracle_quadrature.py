"""Pins for oracle.gl_nodes_weights and the per-order orthonormality that the
butterfly relies on."""

import math

import numpy as np
import pytest
from scipy import special

import oracle
from tests._exact import gl_root_and_weight


@pytest.mark.parametrize("npts", [1, 2, 3, 4, 8, 17, 64])
def test_nodes_match_numpy_leggauss(npts):
    """Library routine: numpy.polynomial.legendre.leggauss (its weights are
    themselves only accurate to ~1e-12 at n ~ 100, so it pins small n only)."""
    x, w = oracle.gl_nodes_weights(npts)
    xr, wr = np.polynomial.legendre.leggauss(npts)
    np.testing.assert_allclose(x, xr, atol=2e-16 * max(1, npts))
    np.testing.assert_allclose(w, wr, rtol=2e-14 * npts)


@pytest.mark.parametrize("npts", [100, 2048])
def test_nodes_and_weights_in_extended_precision(npts):
    """The definition of Section 2, eq. thetas solved in 40-digit arithmetic:
    Newton on P_n from the oracle's node, then w = 2/((1-x^2) P_n'(x)^2) at the
    refined root.  Nodes to ~1 ulp; weights to n * 2e-15 relative (the degree
    recurrence's roundoff near the poles bounds the double-precision angle)."""
    xo, wo = oracle.gl_nodes_weights(npts)
    n = npts
    for i in sorted({0, 1, 7, n // 3, n // 2, n - 2, n - 1}):
        x, w = gl_root_and_weight(n, float(xo[i]), digits=40, steps=4)
        assert abs(xo[i] - float(x)) <= 1.2e-16
        assert abs(wo[i] / float(w) - 1) <= 2e-15 * n, (i, wo[i], float(w))


def test_closed_form_nodes():
    """Textbook closed forms: n = 2: +-1/sqrt 3, w = 1; n = 4:
    x = +-sqrt(3/7 -+ (2/7) sqrt(6/5)), w = (18 +- sqrt 30)/36."""
    x, w = oracle.gl_nodes_weights(2)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], rtol=1e-15)
    np.testing.assert_allclose(w, [1, 1], rtol=1e-15)
    x, w = oracle.gl_nodes_weights(4)
    a = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))
    b = math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
    np.testing.assert_allclose(x, [-b, -a, a, b], rtol=1e-15)
    wa = (18 + math.sqrt(30)) / 36
    wb = (18 - math.sqrt(30)) / 36
    np.testing.assert_allclose(w, [wb, wa, wa, wb], rtol=1e-14)


@pytest.mark.parametrize("l", [4, 64, 512, 1024])
def test_nodes_are_zeros_of_P2l_and_rule_is_exact(l):
    """Section 2, eq. thetas: the 2l nodes are the zeros of P-bar^0_{2l}
    (scipy's P_{2l} vanishes there, relative to its derivative), sum w = 2, and
    the rule integrates x^{2j} exactly for 2j <= 4l - 1."""
    x, w = oracle.gl_nodes_weights(2 * l)
    assert np.all(np.diff(x) > 0)
    n = 2 * l
    p = special.eval_legendre(n, x)
    dp = n * (x * p - special.eval_legendre(n - 1, x)) / (x * x - 1)
    assert np.max(np.abs(p / dp)) < 5e-16 * n
    assert abs(w.sum() - 2) < 1e-13
    for j in range(0, 2 * l, max(1, l // 8)):
        assert abs(np.sum(w * x ** (2 * j)) - 2 / (2 * j + 1)) < 1e-14 * max(1, l / 64)


@pytest.mark.parametrize("l", [8, 64, 700])
def test_paper_weights_at_m0_equal_twice_gl_weights(l):
    """Section 2.3, eq. weights1 with m = 0 and n = l: the positive zeros of
    P-bar^0_{2l} are the positive GL nodes and rho_j = 2 w_j; the paper's
    Gauss-Jacobi rule (eq. Christoffel_definition, m = 0) is then exact on even
    monomials of degree <= 4n - 2 over the n positive nodes alone.  The
    derivative of P-bar^0_{2l} comes from scipy's P_{2l}, P_{2l-1}."""
    x, w = oracle.gl_nodes_weights(2 * l)
    xp, wp = x[l:], w[l:]
    n2 = 2 * l
    dP = n2 * (xp * special.eval_legendre(n2, xp) - special.eval_legendre(n2 - 1, xp)) / (xp * xp - 1)
    dPbar = math.sqrt((2 * n2 + 1) / 2) * dP
    rho = 2 * (0 + 4 * l + 1) / ((1 - xp * xp) * dPbar * dPbar)
    # pointwise, where evaluating the formula at the rounded node is well
    # conditioned (its relative sensitivity is ~ 2 dx / (1 - x^2))
    ok = (1 - xp * xp) > 0.05
    np.testing.assert_allclose(rho[ok], 2 * wp[ok], rtol=1e-12)
    for j in range(0, 2 * l, max(1, l // 4)):
        assert abs(np.sum(rho * xp ** (2 * j)) - 2 / (2 * j + 1)) < 1e-13 * max(1, l / 64)


@pytest.mark.parametrize("l,ms", [(16, None), (64, range(0, 128, 5)), (512, [0, 1, 2, 511, 512, 1000, 1023])])
def test_unit_matrices_have_orthonormal_columns(l, ms):
    """Section 4, eqs. transform/transform2 (GL form): the parity-split weighted
    blocks sqrt(2 w_i) P-bar^m_{m+p+2j}(x_i) over the positive nodes have
    orthonormal columns (discrete orthonormality of each order under GL
    quadrature, folded by the parity of Section 2.3)."""
    for m in (range(2 * l) if ms is None else ms):
        for p in (0, 1):
            A = oracle.unit_matrix(l, m, p)
            if A.shape[1] == 0:
                continue
            assert A.shape == (l, (2 * l - m - p + 1) // 2)
            # roundoff: length-l dot products of values from a degree-2l recurrence
            np.testing.assert_allclose(A.T @ A, np.eye(A.shape[1]), atol=2e-14 + 2.5e-16 * l)
