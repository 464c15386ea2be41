"""Gauss-Legendre nodes/weights and normalized associated Legendre functions.

Test infrastructure only (see ``oracle/__init__.py``).  Plain float64 numpy.

Definitions followed:

* Section 2, eq. thetas: the 2l values cos(theta_k) are the zeros of
  P-bar^0_{2l}, i.e. the Gauss-Legendre nodes of degree 2l, ascending.
* Section 2.3, eq. association: P-bar^m_l(x) =
  sqrt((2l+1)/2 * (l-m)!/(l+m)!) (1-x^2)^{m/2} d^m/dx^m P_l(x), with no
  Condon-Shortley sign; orthonormal on (-1, 1) for fixed m.
* Section 4 (evaluation by recurrence): values are produced by a three-term
  recurrence and underflow is countered by tracking exponents explicitly.
  The oracle deliberately uses the classical recurrence in x (degree k ->
  k+1), NOT the x^2 recurrence of eq. recurrence that the product uses, so
  the two cross-validate.
"""

import numpy as np

# Rescale the running mantissas whenever they leave [2^-RESCALE, 2^RESCALE].
_RESCALE = 600


def gl_nodes_weights(npts):
    """Zeros x_0 < ... < x_{npts-1} of the Legendre polynomial P_npts and the
    Gauss-Legendre weights w_i = 2 / ((1 - x_i^2) P'_npts(x_i)^2).

    Section 2, eq. thetas (with npts = 2l).  Newton's method on
    P_npts(cos theta) in the angle theta, started from
    theta = pi (i + 3/4) / (npts + 1/2).  P_n is evaluated with the textbook
    recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1} at the rounded
    x~ = fl(cos theta), then carried to the exact cos theta by one Taylor term,
    with delta = cos theta - x~ computed without cancellation from the
    half-angle identity and P'' from Legendre's equation
    (1-x^2) P'' = 2x P' - n(n+1) P (eq. sturm-liouville_Leg at m = 0).
    Near x = +-1 both the node angle and the weight are ill-conditioned in the
    rounded x (relative sensitivity ~ 2 dx / (1 - x^2)); this keeps them
    accurate to a few ulp.
    """
    n = int(npts)
    if n < 1:
        raise ValueError("npts must be >= 1")
    i = np.arange(n, dtype=np.float64)
    theta = np.pi * (i + 0.75) / (n + 0.5)

    def p_and_dp_at_cos(theta):
        xr = np.cos(theta)
        north = theta <= np.pi / 2
        # delta = cos(theta) - xr, via cos = 1 - 2 sin^2(t/2) = -1 + 2 cos^2(t/2)
        delta = np.where(north,
                         (1.0 - xr) - 2.0 * np.sin(theta / 2) ** 2,
                         2.0 * np.cos(theta / 2) ** 2 - (1.0 + xr))
        pn, pn1 = _legendre_p_pair(n, xr)
        one_m_x2 = (1.0 - xr) * (1.0 + xr)
        dp = n * (pn1 - xr * pn) / one_m_x2          # (1-x^2) P' = n (P_{n-1} - x P_n)
        d2p = (2.0 * xr * dp - n * (n + 1.0) * pn) / one_m_x2
        return xr, pn + dp * delta, dp + d2p * delta

    for _ in range(100):
        _, p, dp = p_and_dp_at_cos(theta)
        dtheta = p / (np.sin(theta) * dp)  # d/dtheta P(cos theta) = -sin(theta) P'
        theta = theta + dtheta
        if np.max(np.abs(dtheta)) < 1e-18:
            break
    x, _, dp = p_and_dp_at_cos(theta)
    s = np.sin(theta)
    w = 2.0 / (s * s * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def _legendre_p_pair(n, x):
    """(P_n(x), P_{n-1}(x)) for the unnormalized Legendre polynomials."""
    p_prev = np.zeros_like(x)
    p = np.ones_like(x)
    for j in range(n):
        p_prev, p = p, ((2 * j + 1) * x * p - j * p_prev) / (j + 1)
    return p, p_prev


def _degree_walk(m, x, kmax):
    """Yields (k, mantissa of P-bar^m_k, mantissa of P-bar^m_{k-1}, exponent)
    for k = m..kmax: the values are ldexp(mantissa, exponent) with the one
    exponent per node that the two live mantissas share (legendre_table)."""
    s = np.sqrt((1.0 - x) * (1.0 + x))

    # diagonal P-bar^m_m with its own exponent per node
    mant = np.full(x.shape, 1.0 / np.sqrt(2.0))
    expo = np.zeros(x.shape, dtype=np.int64)
    for j in range(1, m + 1):
        mant = mant * (np.sqrt((2.0 * j + 1.0) / (2.0 * j)) * s)
        mant, e = np.frexp(mant)
        expo += e
    p_prev = np.zeros_like(mant)
    yield m, mant, p_prev, expo
    p_cur = mant
    a_prev = None
    for k in range(m, kmax):
        kk = k + 1.0
        a_next = np.sqrt((4.0 * kk * kk - 1.0) / ((kk - m) * (kk + m)))
        if a_prev is None:
            p_next = a_next * x * p_cur
        else:
            p_next = a_next * x * p_cur - (a_next / a_prev) * p_prev
        a_prev = a_next
        p_prev, p_cur = p_cur, p_next
        # common rescale of the two live mantissas of each node
        big = np.maximum(np.abs(p_prev), np.abs(p_cur))
        need = (big > 2.0 ** _RESCALE) | ((big < 2.0 ** -_RESCALE) & (big > 0.0))
        if np.any(need):
            _, sh = np.frexp(np.where(need, big, 1.0))
            sh = np.where(need, sh, 0)
            p_prev = np.ldexp(p_prev, -sh)
            p_cur = np.ldexp(p_cur, -sh)
            expo = expo + sh
        yield k + 1, p_cur, p_prev, expo


def legendre_table(m, x, kmax):
    """P-bar^m_k(x) for k = m..kmax, as an array of shape (kmax - m + 1, len(x)).

    Section 2.3, eq. association.  Evaluation:

    * diagonal: P-bar^0_0 = 1/sqrt(2) and
      P-bar^j_j = sqrt((2j+1)/(2j)) sqrt(1-x^2) P-bar^{j-1}_{j-1};
    * degree recurrence for fixed m:
      P-bar^m_{k+1} = a_{k+1} x P-bar^m_k - (a_{k+1}/a_k) P-bar^m_{k-1},
      a_k = sqrt((4k^2 - 1)/(k^2 - m^2)) (the second term is absent for k = m);
    * every node carries (mantissa, binary exponent); the mantissas are
      renormalized whenever they leave [2^-600, 2^600], and values are
      converted with ldexp at the end (flushing to 0 below the float64 range),
      as Section 4 prescribes for countering underflow.
    """
    m = int(m)
    kmax = int(kmax)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    if m < 0 or kmax < m:
        return np.zeros((0, x.size))
    out = np.zeros((kmax - m + 1, x.size))
    for k, mant, _, expo in _degree_walk(m, x, kmax):
        out[k - m] = np.ldexp(mant, expo)
    return out


def legendre_top_pair(m, N, x):
    """P-bar^m_N(x) and P-bar^m_{N-1}(x) by the recurrence of legendre_table,
    keeping only the last two degrees: (mantissa_N, mantissa_{N-1},
    exponent), the values being ldexp(mantissa, exponent) (N >= m + 1)."""
    m, N = int(m), int(N)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    if N < m + 1:
        raise ValueError("N must exceed m")
    for _, cur, prev, expo in _degree_walk(m, x, N):
        pass
    return cur, prev, expo


def legendre_value(m, k, x):
    """P-bar^m_k(x) (Section 2.3, eq. association) for scalar or array x."""
    return legendre_table(m, x, k)[-1]
