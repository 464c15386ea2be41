"""Pins for oracle.sht: brute force of eq. expansion, round trips, special
fields, the phi stage against numpy.fft, and the parity split."""

import cmath
import math

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import inputs
from tests._exact import pbar_exact


def _brute_synthesis(beta, l):
    """Section 2, eq. expansion summed term by term over k and m = -k..k, with
    P-bar from its definition (exact polynomials) and beta^{-m} = conj(beta^m)."""
    off = oracle.triangle_offsets(l)
    x, _ = np.polynomial.legendre.leggauss(2 * l)  # library nodes, not the oracle's
    phis = [2 * math.pi * (j + 0.5) / (4 * l - 1) for j in range(4 * l - 1)]
    pb = {}
    for k in range(2 * l):
        for m in range(k + 1):
            pb[(m, k)] = [float(pbar_exact(m, k, xi)) for xi in x]
    f = np.zeros((2 * l, 4 * l - 1))
    for i in range(2 * l):
        for j, ph in enumerate(phis):
            acc = 0j
            for k in range(2 * l):
                for m in range(-k, k + 1):
                    b = beta[off[abs(m)] + k - abs(m)]
                    if m < 0:
                        b = b.conjugate()
                    acc += b * pb[(abs(m), k)][i] * cmath.exp(1j * m * ph)
            assert abs(acc.imag) < 1e-12
            f[i, j] = acc.real
    return f


@pytest.mark.parametrize("l", [1, 2, 4])
def test_brute_force_synthesis(l):
    beta = inputs.random_beta(l, seed=100 + l)
    np.testing.assert_allclose(oracle.sht_synthesis(beta, l), _brute_synthesis(beta, l), atol=1e-13)


@pytest.mark.slow
def test_brute_force_synthesis_l8():
    l = 8
    beta = inputs.random_beta(l, seed=108)
    np.testing.assert_allclose(oracle.sht_synthesis(beta, l), _brute_synthesis(beta, l), atol=5e-13)


@pytest.mark.parametrize("l", [3, 16, 64])
def test_round_trip(l):
    """Analysis inverts synthesis exactly (up to roundoff) on band-limited
    fields: GL quadrature with 2l nodes is exact for the products of degree <=
    4l-2, and 4l-1 phis resolve |m| <= 2l-1 (Section 2)."""
    beta = inputs.random_beta(l, seed=l)
    f = oracle.sht_synthesis(beta, l)
    back = oracle.sht_analysis(f, l)
    np.testing.assert_allclose(back, beta, atol=1e-13 * math.sqrt(l))
    G = oracle.legendre_synthesis(beta, l)
    np.testing.assert_allclose(oracle.legendre_analysis(G, l), beta, atol=1e-13 * math.sqrt(l))


def test_special_fields():
    """f = 1 has beta^0_0 = sqrt 2 (P-bar^0_0 = 1/sqrt 2); f = cos(theta) has
    beta^0_1 = sqrt(2/3) (P-bar^0_1 = sqrt(3/2) x); all else 0."""
    l = 6
    x, _ = oracle.gl_nodes_weights(2 * l)
    N = 4 * l - 1
    b = oracle.sht_analysis(np.ones((2 * l, N)), l)
    ref = np.zeros_like(b)
    ref[0] = math.sqrt(2)
    np.testing.assert_allclose(b, ref, atol=1e-14)
    b = oracle.sht_analysis(np.repeat(x[:, None], N, axis=1), l)
    ref = np.zeros_like(b)
    ref[1] = math.sqrt(2 / 3)
    np.testing.assert_allclose(b, ref, atol=1e-14)


def test_phi_stage_against_numpy_fft():
    """Library routine: G^m_i = (1/N) e^{-i pi m / N} FFT(f_i)_m, because
    phi_j = 2 pi (j + 1/2)/N (Section 2, eq. phis)."""
    l = 10
    N = 4 * l - 1
    rng = np.random.default_rng(5)
    f = rng.standard_normal((2 * l, N))
    G = oracle.phi_analysis(f, l)
    F = np.fft.fft(f, axis=1)[:, : 2 * l].T
    ref = F * np.exp(-1j * np.pi * np.arange(2 * l) / N)[:, None] / N
    np.testing.assert_allclose(G, ref, atol=1e-14)
    # synthesis: real inverse FFT of the Hermitian spectrum built from G
    spec = np.zeros((2 * l, N), dtype=complex)
    H = (G * np.exp(1j * np.pi * np.arange(2 * l) / N)[:, None]).T
    spec[:, : 2 * l] = H
    spec[:, N - 2 * l + 1:] = np.conj(H[:, 1:][:, ::-1])
    np.testing.assert_allclose(oracle.phi_synthesis(G, l), np.real(np.fft.ifft(spec, axis=1)) * N, atol=1e-12)


def test_single_mode():
    """f = cos(m0 phi) has G^{m0} = 1/2 and no other mode (exactness of the
    4l-1 point rule)."""
    l = 5
    ph = oracle.phis(l)
    for m0 in range(2 * l):
        f = np.repeat(np.cos(m0 * ph)[None, :], 2 * l, axis=0)
        G = oracle.phi_analysis(f, l)
        ref = np.zeros_like(G)
        ref[m0] = 1.0 if m0 == 0 else 0.5
        np.testing.assert_allclose(G, ref, atol=1e-14)


def test_parity_split_reassembles_legendre_stage():
    """Section 2.3 parity + Section 4 weights: G^m(x_{l+i}) = E_i + O_i and
    G^m(x_{l-1-i}) = E_i - O_i, with E = A^{m,0} beta_even / sqrt(2w) and
    O = A^{m,1} beta_odd / sqrt(2w) from the per-unit blocks."""
    l = 12
    beta = inputs.random_beta(l, seed=3)
    G = oracle.legendre_synthesis(beta, l)
    off = oracle.triangle_offsets(l)
    x, w = oracle.gl_nodes_weights(2 * l)
    s = np.sqrt(2 * w[l:])
    for m in range(2 * l):
        bm = beta[off[m]:off[m + 1]]
        E = oracle.unit_matrix(l, m, 0) @ bm[0::2] / s
        O = oracle.unit_matrix(l, m, 1) @ bm[1::2] / s if len(bm) > 1 else 0
        np.testing.assert_allclose(G[m, l:], E + O, atol=1e-13)
        np.testing.assert_allclose(G[m, :l][::-1], E - O, atol=1e-13)


def test_analysis_is_weighted_adjoint():
    """legendre_analysis(G) = legendre_adjoint(w G) and <synth b, g> =
    <b, adjoint g> (real inner product, complex as 2 reals)."""
    l = 9
    rng = np.random.default_rng(9)
    G = rng.standard_normal((2 * l, 2 * l)) + 1j * rng.standard_normal((2 * l, 2 * l))
    _, w = oracle.gl_nodes_weights(2 * l)
    np.testing.assert_allclose(oracle.legendre_analysis(G, l), oracle.legendre_adjoint(G * w, l), atol=1e-14)
    b = inputs.random_beta(l, seed=4)
    lhs = np.vdot(oracle.legendre_synthesis(b, l), G).real
    rhs = np.vdot(b, oracle.legendre_adjoint(G, l)).real
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_loss_gradient_against_central_differences():
    """The gradient convention of the differentiable synthesis: for
    L(beta) = sum |synth(beta) - g|^2 over all orders and nodes, the gradient
    dL/dRe beta + i dL/dIm beta equals 2 adjoint(synth(beta) - g).  Pinned by
    central differences of L itself on every real coordinate; L is quadratic,
    so the differences are exact up to rounding."""
    l = 4
    beta = inputs.random_beta(l, seed=21, decay=True)
    g = oracle.legendre_synthesis(inputs.random_beta(l, seed=22), l)

    def loss(b):
        return float(np.sum(np.abs(oracle.legendre_synthesis(b, l) - g) ** 2))

    grad = 2.0 * oracle.legendre_adjoint(oracle.legendre_synthesis(beta, l) - g, l)
    ms, _ = inputs.triangle_index(l)
    h = 1e-6
    fd = np.zeros_like(beta)
    for c in range(beta.size):
        for unit in (1.0, 1j):
            if unit == 1j and ms[c] == 0:
                continue  # beta^0_k is real: no imaginary coordinate
            e = np.zeros_like(beta)
            e[c] = h * unit
            d = (loss(beta + e) - loss(beta - e)) / (2 * h)
            fd[c] += d * unit
    assert np.all(grad.imag[ms == 0] == 0.0)
    np.testing.assert_allclose(fd, grad, rtol=0, atol=1e-7 * np.abs(grad).max())
