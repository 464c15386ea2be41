"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

Holds none of the transform's arithmetic: only random draws and the storage
layout of the coefficient triangle.

* ``random_beta``: coefficients beta^m_k of a real field (m >= 0 stored),
  Re and Im iid N(0, 1) (Im = 0 at m = 0), optionally scaled by 1/(k+1),
  m-major triangle (beta^m_k at offset(m) + k - m, offset(m) =
  sum_{m' < m} (2l - m')).
* ``random_grid``: a real band-limited-free random grid (used for adjoint
  and analysis checks that do not need band-limited data).
"""

import numpy as np


def triangle_size(l):
    L = 2 * int(l)
    return L * (L + 1) // 2


def triangle_index(l):
    """(m, k) of every triangle slot, in storage order."""
    L = 2 * int(l)
    ms = np.concatenate([np.full(L - m, m) for m in range(L)])
    ks = np.concatenate([np.arange(m, L) for m in range(L)])
    return ms, ks


def random_beta(l, seed, decay=False, dtype=np.complex128):
    """beta^m_k iid complex N(0, 1) (real for m = 0), times 1/(k+1) if ``decay``."""
    rng = np.random.default_rng(seed)
    n = triangle_size(l)
    re = rng.standard_normal(n)
    im = rng.standard_normal(n)
    ms, ks = triangle_index(l)
    im[ms == 0] = 0.0
    beta = re + 1j * im
    if decay:
        beta = beta / (ks + 1.0)
    return beta.astype(dtype)


def random_grid(l, seed, dtype=np.float64):
    """Real values on the (2l) x (4l-1) grid, iid N(0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((2 * int(l), 4 * int(l) - 1)).astype(dtype)


def random_G(l, seed, dtype=np.complex128):
    """Complex Legendre-stage values G[m][i], (2l, 2l), iid complex N(0, 1)."""
    rng = np.random.default_rng(seed)
    L = 2 * int(l)
    return (rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))).astype(dtype)
