"""The interpolative decomposition of Section 2.1 (eq. 2.1, Remark
QR_algorithm) as the builders compute it (sht_interp_decomp, host only),
checked against singular values from numpy:

  * structure: the skeleton and redundant columns partition the columns, the
    redundant ones in ascending order;
  * the strong rank-revealing bound: every interpolation coefficient is at
    most 2 in magnitude;
  * accuracy: ||A[:, red] - A[:, skel] T||_2 <= sqrt(4 k (n - k) + 1)
    sigma_{k+1}(A), the bound of a strong rank-revealing QR with f = 2;
  * the rank rule: sigma_{k+1}(A) <= sqrt(n - k) eps, since every remaining
    column norm is at most eps when the QR stops.

The Kahan matrix is the classic case where column pivoting alone does not
reveal the rank: there the exchange step must fire and bring the error down
to the order of sigma_{k+1}."""

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import sht


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def check_id(A, eps, expect_swaps=None):
    h, w = A.shape
    skel, red, T, swaps = sht.interp_decomp(A, eps)
    k = len(skel)
    assert sorted(np.concatenate([skel, red]).tolist()) == list(range(w))
    assert np.all(np.diff(red) > 0)
    assert T.shape == (k, w - k)
    if T.size:
        assert np.abs(T).max() <= 2.0 + 1e-12
    sv = np.linalg.svd(A, compute_uv=False)
    if k < w:
        sk1 = sv[k] if k < len(sv) else 0.0
        err = np.linalg.norm(A[:, red] - A[:, skel] @ T, 2)
        assert err <= np.sqrt(4 * k * (w - k) + 1) * sk1 * (1 + 1e-6) + 1e-13 * sv[0], (err, sk1)
        assert sk1 <= np.sqrt(w - k) * eps * (1 + 1e-9)
    if expect_swaps is not None:
        assert swaps >= expect_swaps
    return k, swaps


@pytest.mark.parametrize("h,w,decay", [(60, 40, 0.7), (200, 64, 0.5), (40, 60, 0.8), (128, 32, 0.9)])
def test_random_matrices_with_decaying_spectrum(h, w, decay):
    rng = np.random.default_rng(h * 1000 + w)
    r = min(h, w)
    eps = decay ** (r // 2)  # cuts the spectrum about half way
    U, _ = np.linalg.qr(rng.standard_normal((h, r)))
    V, _ = np.linalg.qr(rng.standard_normal((w, r)))
    A = (U * decay ** np.arange(r)) @ V.T
    k, _ = check_id(A, eps)
    assert 0 < k < r  # the threshold cuts the spectrum


@pytest.mark.parametrize("n,c", [(40, 0.6), (30, 0.7), (50, 0.65)])
def test_kahan_matrix_needs_the_exchange_step(n, c):
    s = np.sqrt(1.0 - c * c)
    R = np.eye(n) - c * np.triu(np.ones((n, n)), 1)
    K = np.diag(s ** np.arange(n)) @ R
    K = K * (1.0 - 1e-10 * np.arange(n))[None, :]  # column pivoting keeps the natural order
    eps = 1.2 * s ** (n - 1)  # pivoted QR alone stops one column short, residual s^(n-1)
    k, swaps = check_id(K, eps, expect_swaps=1)
    assert k < n
    skel, red, T, _ = sht.interp_decomp(K, eps)
    err = np.linalg.norm(K[:, red] - K[:, skel] @ T, 2)
    sv = np.linalg.svd(K, compute_uv=False)
    # the exchanges take the error from s^(n-1) down to the order of sigma_n
    assert err < 0.5 * s ** (n - 1) and err <= np.sqrt(4 * k * (n - k) + 1) * sv[k] * (1 + 1e-6) + 1e-13


@pytest.mark.parametrize("l,m,p", [(32, 0, 0), (32, 5, 1), (48, 20, 0)])
def test_weighted_gauss_legendre_blocks(l, m, p):
    """Blocks of the matrices the butterflies compress (the oracle's weighted
    Gauss-Legendre parity blocks), split into row halves as the merges do."""
    A = oracle.unit_matrix(l, m, p)
    for eps in (1e-12, 1e-6):
        check_id(A[: l // 2], eps)
        check_id(A[l // 2:], eps)
        check_id(A, eps)


def test_invalid_arguments():
    import ctypes
    L = sht.lib()
    k = ctypes.c_int()
    buf = np.zeros(16)
    perm = np.zeros(4, dtype=np.int32)
    A = np.ones((4, 4))
    for h, w, eps in [(0, 4, 1e-6), (4, 0, 1e-6), (4, 4, 0.0), (4, 70000, 1e-6)]:
        assert L.sht_interp_decomp(A.ctypes.data, h, w, eps, ctypes.byref(k), perm.ctypes.data,
                                   buf.ctypes.data, None) == 1
