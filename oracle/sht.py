"""Direct O(l^3) spherical harmonic transform on the Gauss-Legendre grid.

Test infrastructure only (see ``oracle/__init__.py``).  Plain float64 /
complex128 numpy; matrix products use the library matmul, nothing is fused.

Data layout shared with the product's C-ABI (a data format, not arithmetic):

* beta: complex coefficients of a real field, m >= 0 only, stored m-major as a
  triangle: beta^m_k at ``triangle_offsets(l)[m] + (k - m)`` for
  k = m..2l-1, m = 0..2l-1 (2l(2l+1)/2 entries).  beta^{-m}_k =
  conj(beta^m_k) is implied, and beta^0_k is real.
* G: the Legendre-stage values G^m(x_i) = sum_k beta^m_k P-bar^m_k(x_i),
  a (2l, 2l) complex array [m][i], nodes ascending.
* f: real grid values f(theta_i, phi_j), a (2l, 4l-1) array [i][j].
"""

import numpy as np

from .legendre import gl_nodes_weights, legendre_table


def triangle_offsets(l):
    """offset(m) = sum_{m' < m} (2l - m') for m = 0..2l-1, plus the total size
    2l(2l+1)/2 as the last entry (Section 2, eq. expansion: degrees k < 2l)."""
    L = 2 * int(l)
    counts = L - np.arange(L)
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


def phis(l):
    """phi_j = 2 pi (j + 1/2) / (4l - 1), j = 0..4l-2 (Section 2, eq. phis)."""
    N = 4 * int(l) - 1
    return 2.0 * np.pi * (np.arange(N) + 0.5) / N


def legendre_synthesis(beta, l, orders=None):
    """G^m(x_i) = sum_{k=m}^{2l-1} beta^m_k P-bar^m_k(x_i) at all 2l
    Gauss-Legendre nodes (the sums over k of Section 2, eq.
    alternate_expansion).  Returns G (2l, 2l) complex; with ``orders`` only
    those rows m are computed (the others stay zero)."""
    l = int(l)
    L = 2 * l
    beta = np.asarray(beta, dtype=np.complex128)
    off = triangle_offsets(l)
    x, _ = gl_nodes_weights(L)
    G = np.zeros((L, L), dtype=np.complex128)
    for m in (range(L) if orders is None else orders):
        P = legendre_table(m, x, L - 1)  # (2l - m, 2l)
        G[m] = beta[off[m]:off[m + 1]] @ P
    return G


def legendre_analysis(G, l, orders=None):
    """beta^m_k = sum_i w_i P-bar^m_k(x_i) G^m(x_i): the Gauss-Legendre
    quadrature that inverts the Legendre stage for band-limited data
    (Section 2: the forward transform, the transpose of the sums over k)."""
    l = int(l)
    L = 2 * l
    G = np.asarray(G, dtype=np.complex128)
    off = triangle_offsets(l)
    x, w = gl_nodes_weights(L)
    beta = np.zeros(off[-1], dtype=np.complex128)
    for m in (range(L) if orders is None else orders):
        P = legendre_table(m, x, L - 1)
        beta[off[m]:off[m + 1]] = P @ (w * G[m])
    return beta


def legendre_adjoint(Ghat, l, orders=None):
    """The transpose of legendre_synthesis without quadrature weights:
    beta-hat^m_k = sum_i P-bar^m_k(x_i) G-hat^m(x_i)."""
    l = int(l)
    L = 2 * l
    Ghat = np.asarray(Ghat, dtype=np.complex128)
    off = triangle_offsets(l)
    x, _ = gl_nodes_weights(L)
    beta = np.zeros(off[-1], dtype=np.complex128)
    for m in (range(L) if orders is None else orders):
        P = legendre_table(m, x, L - 1)
        beta[off[m]:off[m + 1]] = P @ Ghat[m]
    return beta


def _phase_matrix(l):
    """E[m, j] = exp(i m phi_j), m = 0..2l-1, j = 0..4l-2."""
    L = 2 * int(l)
    return np.exp(1j * np.outer(np.arange(L), phis(l)))


def phi_synthesis(G, l):
    """f(theta_i, phi_j) = sum_{m=-(2l-1)}^{2l-1} G^m_i e^{i m phi_j} for a real
    field (G^{-m} = conj(G^m)), i.e. Re G^0_i + 2 Re sum_{m>=1} G^m_i e^{i m phi_j}
    (the sums over m of Section 2, eq. alternate_expansion, as a naive DFT)."""
    L = 2 * int(l)
    G = np.asarray(G, dtype=np.complex128)
    c = np.full(L, 2.0)
    c[0] = 1.0
    return np.real((c[:, None] * G).T @ _phase_matrix(l))


def phi_analysis(f, l):
    """G^m_i = (1/(4l-1)) sum_j f(theta_i, phi_j) e^{-i m phi_j}, m = 0..2l-1:
    exact for band-limited f because the 4l-1 equispaced phis of eq. phis
    resolve all 4l-1 frequencies |m| <= 2l-1."""
    N = 4 * int(l) - 1
    f = np.asarray(f, dtype=np.float64)
    return (np.conj(_phase_matrix(l)) @ f.T) / N


def sht_synthesis(beta, l):
    """Full inverse SHT of Section 2, eq. expansion on the tensor-product grid:
    beta -> f (2l, 4l-1)."""
    return phi_synthesis(legendre_synthesis(beta, l), l)


def sht_analysis(f, l):
    """Full forward SHT of Section 2: f (2l, 4l-1) -> beta."""
    return legendre_analysis(phi_analysis(f, l), l)


def unit_matrix(l, m, p):
    """The parity-split, weighted Legendre block used by the butterfly:
    A[i, j] = sqrt(2 w_{l+i}) P-bar^m_{m+p+2j}(x_{l+i}) over the l positive
    nodes x_{l+i} (i = 0..l-1, ascending), j = 0..n-1 with
    n = ceil((2l - m - p)/2).  This is the Gauss-Legendre form of the
    unitary per-order map of Section 4, eq. transform (p = 0) and eq.
    transform2 (p = 1); its columns are orthonormal."""
    l = int(l)
    L = 2 * l
    x, w = gl_nodes_weights(L)
    xp = x[l:]
    wp = w[l:]
    n = max(0, (L - m - p + 1) // 2)
    if n == 0:
        return np.zeros((l, 0))
    P = legendre_table(m, xp, L - 1)  # rows k = m..2l-1
    rows = P[p::2][:n]  # degrees m+p, m+p+2, ...
    return (np.sqrt(2.0 * wp)[:, None] * rows.T).copy()
