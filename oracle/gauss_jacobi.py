"""The paper's own per-order matrices (Section 4): Gauss-Jacobi-type nodes,
the weights of Lemma quadratures, and the direct transforms of eqs.
transform and transform2.

Test infrastructure only (see ``oracle/__init__.py``).  Plain float64 numpy.

* Nodes (Lemma distinct_theorem): the n zeros in (0, 1) of P-bar^m_N with
  N = m + 2n (parity 0, eq. zeros) or N = m + 2n + 1 (parity 1, eq. zeros2).
  Found by sign changes of P-bar^m_N(cos theta) on a grid of angles, then
  bisection in theta to the last bit and two Newton steps in x; P-bar is
  evaluated with this package's classical three-term recurrence in x
  (``legendre_top_pair``).
  Nothing here uses the x^2 recurrence or its Jacobi matrix, which the
  product's nodes come from.
* Weights: eq. weights1 (parity 0) and eq. weights2 (parity 1), both
  w_j = 2 (2N + 1) / ((1 - x_j^2) P-bar'^m_N(x_j)^2), and eq. weights2_0,
  sigma_n = (2N + 1) / P-bar'^m_N(0)^2.  The derivative comes from the
  textbook identity
  (1 - x^2) P-bar'^m_N = sqrt((2N + 1)(N^2 - m^2) / (2N - 1)) P-bar^m_{N-1}
  - N x P-bar^m_N.
* Transforms: A[i, j] = sqrt(w_i) P-bar^m_{m+p+2j}(x_i) (eq. transform for
  p = 0, eq. transform2 for p = 1); the forward map is A beta and the
  inverse map its transpose (A is orthogonal by Lemma quadratures).
"""

import numpy as np

from .legendre import legendre_table, legendre_top_pair


def _values(m, N, x):
    """P-bar^m_N(x) and P-bar^m_{N-1}(x) as floats, and the sign of the
    first (exact also where the value underflows)."""
    cur, prev, expo = legendre_top_pair(m, N, x)
    return np.ldexp(cur, expo), np.ldexp(prev, expo), np.sign(cur)


def _derivative(m, N, x):
    """P-bar'^m_N(x) from the identity in the module docstring."""
    pn, pn1, _ = _values(m, N, x)
    c = np.sqrt((2.0 * N + 1.0) * (N * N - m * m) / (2.0 * N - 1.0))
    return (c * pn1 - N * x * pn) / ((1.0 - x) * (1.0 + x))


def gj_nodes_weights(m, parity, n):
    """(x, w): the n positive zeros x_0 < ... < x_{n-1} of P-bar^m_N,
    N = m + 2n + parity, and their weights (rho_j of eq. weights1 for
    parity 0, sigma_j of eq. weights2 for parity 1)."""
    m, parity, n = int(m), int(parity), int(n)
    if m < 0 or n < 1 or parity not in (0, 1):
        raise ValueError("need m >= 0, n >= 1, parity 0 or 1")
    N = m + 2 * n + parity
    # angles in (0, pi/2), finer than the zero spacing (about pi / N)
    G = 16 * N + 64
    theta = 0.5 * np.pi * (np.arange(G) + 0.5) / G
    _, _, sg = _values(m, N, np.cos(theta))
    ch = np.nonzero(sg[:-1] * sg[1:] < 0)[0]
    if ch.size != n:
        raise RuntimeError(f"found {ch.size} sign changes of P-bar^{m}_{N} in (0, 1), expected {n}")
    lo, hi = theta[ch].copy(), theta[ch + 1].copy()
    s_lo = sg[ch]
    for _ in range(64):
        mid = 0.5 * (lo + hi)
        done = (mid <= lo) | (mid >= hi)
        if np.all(done):
            break
        _, _, sm = _values(m, N, np.cos(mid))
        same = sm == s_lo
        lo = np.where(same & ~done, mid, lo)
        hi = np.where(~same & ~done, mid, hi)
    th = 0.5 * (lo + hi)
    x = np.cos(th)[::-1]  # ascending in x
    # the angle is resolved to ~1e-16 absolute, a few hundred ulp of x near
    # x = 0: two Newton steps in x finish the small nodes
    for _ in range(2):
        pn, _, _ = _values(m, N, x)
        x = x - pn / _derivative(m, N, x)
    dp = _derivative(m, N, x)
    w = 2.0 * (2.0 * N + 1.0) / ((1.0 - x) * (1.0 + x) * dp * dp)
    return x, w


def gj_sigma_n(m, n):
    """sigma_n of eq. weights2_0: (2m + 4n + 3) / P-bar'^m_{m+2n+1}(0)^2."""
    N = int(m) + 2 * int(n) + 1
    dp = _derivative(int(m), N, np.zeros(1))[0]
    return (2.0 * N + 1.0) / (dp * dp)


def gj_matrix(m, parity, n, rows=None):
    """A[i, j] = sqrt(w_i) P-bar^m_{m+parity+2j}(x_i), j < n, for the rows
    i in ``rows`` (all n by default): eq. transform (parity 0) or eq.
    transform2 (parity 1)."""
    x, w = gj_nodes_weights(m, parity, n)
    idx = np.arange(n) if rows is None else np.asarray(rows)
    T = legendre_table(m, x[idx], m + parity + 2 * n - 2)  # degrees m .. m+parity+2n-2
    P = T[parity::2]  # degrees m + parity + 2j, j < n
    return np.sqrt(w[idx])[:, None] * P.T


def gj_forward(beta, m, parity, rows=None):
    """alpha_i = sum_j beta_j sqrt(w_i) P-bar^m_{m+parity+2j}(x_i) (eqs.
    transform, transform2); beta may carry trailing columns (several
    vectors), real or complex."""
    beta = np.asarray(beta)
    return gj_matrix(m, parity, beta.shape[0], rows) @ beta


def gj_inverse(alpha, m, parity):
    """beta = A^T alpha, the inverse of gj_forward (A is orthogonal)."""
    alpha = np.asarray(alpha)
    return gj_matrix(m, parity, alpha.shape[0]).T @ alpha
