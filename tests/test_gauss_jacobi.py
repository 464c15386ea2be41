"""The paper's own quadrature and matrices (Section 4: Lemma zeros, Lemma
quadratures, eqs. transform and transform2), built on the host by
sht_gauss_jacobi_nodes and sht_unit_stats_gauss_jacobi.

Pins, none of which uses the product's own arithmetic to check itself:
  - at m = 0 the even nodes are the positive Gauss-Legendre nodes of degree
    2n with rho_i = 2 w_i (the oracle's independent Newton iteration);
  - the rules of Lemma quadratures integrate (1 - x^2)^m x^{2k} exactly
    (closed form: the beta integral B(k + 1/2, m + 1));
  - the nodes are zeros of P-bar^m_{m+p+2n} (the oracle's x recurrence);
  - sqrt(rho_i) P-bar^m_{m+p+2j}(x_i) is orthogonal (the oracle's values);
  - the butterflies of the m = n matrices set beside Tables evens / odds
    (tests/golden/paper_evens_odds_tables.txt).
"""

import math
import os

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import sht

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_evens_odds_tables.txt")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def beta_integral(k, m):
    """int_{-1}^{1} (1 - x^2)^m x^{2k} dx = B(k + 1/2, m + 1)."""
    return math.exp(math.lgamma(k + 0.5) + math.lgamma(m + 1) - math.lgamma(k + m + 1.5))


@pytest.mark.parametrize("n", [1, 7, 60])
def test_m0_even_nodes_are_gauss_legendre(n):
    x, rho = sht.gauss_jacobi_nodes(0, 0, n)
    xg, wg = oracle.gl_nodes_weights(2 * n)
    assert np.all(np.diff(x) > 0)
    assert np.max(np.abs(x - xg[n:])) < 1e-14
    assert np.max(np.abs(rho - 2 * wg[n:]) / (2 * wg[n:])) < 1e-11


@pytest.mark.parametrize("m", [0, 3, 40, 300])
@pytest.mark.parametrize("p", [0, 1])
def test_quadrature_rules_are_exact(m, p):
    """Even rule: sum_i rho_i (1-x_i^2)^m x_i^{2k} exact for 2k <= 4n - 2.
    Odd rule: exact for 2k <= 4n once its node at 0 is added (weight
    sigma_n); for k >= 1 that node contributes nothing."""
    n = 40
    x, rho = sht.gauss_jacobi_nodes(m, p, n)
    assert np.all((x > 0) & (x < 1)) and np.all(rho > 0)
    ks = range(0, 2 * n) if p == 0 else range(1, 2 * n + 1)
    for k in ks:
        q = np.sum(rho * (1 - x ** 2) ** m * x ** (2 * k))
        assert abs(q - beta_integral(k, m)) <= 1e-11 * beta_integral(k, m), k


@pytest.mark.parametrize("m,p,n", [(0, 0, 30), (5, 1, 30), (120, 0, 50), (120, 1, 50)])
def test_nodes_are_zeros_and_matrix_is_orthogonal(m, p, n):
    x, rho = sht.gauss_jacobi_nodes(m, p, n)
    P = oracle.legendre_table(m, x, m + p + 2 * n)  # rows: degrees m .. m+p+2n
    top = P[p + 2 * n]
    scale = np.max(np.abs(P[p:p + 2 * n:2]), axis=0)
    assert np.max(np.abs(top) / scale) < 1e-11
    A = np.sqrt(rho)[:, None] * P[p:p + 2 * n:2].T  # A[i, j] = sqrt(rho_i) P-bar^m_{m+p+2j}(x_i)
    assert np.max(np.abs(A.T @ A - np.eye(n))) < 1e-12


@pytest.mark.parametrize("m,p,n", [(0, 0, 40), (0, 1, 40), (7, 1, 64), (200, 0, 90), (300, 1, 300)])
def test_nodes_and_weights_match_oracle(m, p, n):
    """The product's nodes (eigenvalues of the x^2 Jacobi matrix, Newton on
    the x^2 recurrence) and weights (1 / sum of squares) against the
    oracle's (bisection on the x recurrence, eqs. weights1 / weights2)."""
    x, rho = sht.gauss_jacobi_nodes(m, p, n)
    xo, wo = oracle.gj_nodes_weights(m, p, n)
    assert np.max(np.abs(x - xo)) < 2e-15
    assert np.max(np.abs(rho - wo) / wo) < 1e-12


def test_butterfly_errors_at_id_precision():
    for p in (0, 1):
        s = sht.unit_stats(300, 300, p, eps_id=1e-12, leaf_cols=32, gauss_jacobi=True)
        assert s["n"] == 300 and s["eps_fwd"] < 50e-12 and s["eps_inv"] < 50e-12


@pytest.mark.parametrize("p", [0, 1])
def test_m_equals_n_beside_paper_tables_n1250(p):
    """n = m = 1250, C = 60, IDs to 1e-15.  The ranks follow the printed ones
    from below (average within 20 %), the peak memory of the depth-first
    build is within a factor 2, and both errors are at or below the printed
    ones."""
    ref = None
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if int(f[0]) == p and int(f[1]) == 1250:
            ref = dict(k_max=int(f[3]), k_avg=float(f[4]), m_max=float(f[6]), eps_fwd=float(f[7]),
                       eps_inv=float(f[8]))
    s = sht.unit_stats(1250, 1250, p, eps_id=1e-15, leaf_cols=60, gauss_jacobi=True)
    assert abs(s["k_avg"] - ref["k_avg"]) <= 0.20 * ref["k_avg"], s["k_avg"]
    assert s["k_max"] <= ref["k_max"]
    assert ref["m_max"] / 2 <= s["m_max_words"] <= 2 * ref["m_max"]
    assert s["eps_fwd"] <= ref["eps_fwd"] and s["eps_inv"] <= ref["eps_inv"]


def test_invalid_arguments():
    import ctypes
    x = np.zeros(4)
    L = sht.lib()
    assert L.sht_gauss_jacobi_nodes(-1, 0, 4, x.ctypes.data, x.ctypes.data) == 1
    assert L.sht_gauss_jacobi_nodes(0, 2, 4, x.ctypes.data, x.ctypes.data) == 1
    assert L.sht_gauss_jacobi_nodes(0, 0, 0, x.ctypes.data, x.ctypes.data) == 1
    out = sht.sht_unit_stats()
    assert L.sht_unit_stats_gauss_jacobi(0, 0, 0, 1e-12, None, 1, ctypes.byref(out)) == 1


@pytest.mark.parametrize("n,m,p", [(200, 0, 0), (129, 7, 1), (300, 300, 1)])
def test_single_block_streams_match_oracle_on_host(n, m, p):
    """The level-by-level streams of a single-block plan (sht_gj_plan_create),
    decoded and applied on the host (tests/stream_emulator.py, stage by
    stage), against the oracle's A beta and A^T alpha."""
    from tests.stream_emulator import emulate

    P = sht.GJPlan(n, m, p, eps_id=1e-12, leaf_cols=32, host_only=True)
    A = oracle.gj_matrix(m, p, n)
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)
    tol = {0: 1e-11, 2: 1e-11, 1: 1e-6}
    for prec in (0, 2, 1):
        P.prepare(prec)
        a = emulate(P.stream(prec, 0), P.page_bytes, n, prec, 0, b, plain=True)
        assert np.linalg.norm(a - A @ b) / np.linalg.norm(A @ b) < tol[prec]
        bb = emulate(P.stream(prec, 1), P.page_bytes, n, prec, 1, a, plain=True)
        assert np.linalg.norm(bb - A.T @ a) / np.linalg.norm(b) < tol[prec]
        assert P.launches(prec, 0) >= 3 and P.launches(prec, 1) >= 3
    P.close()


def test_single_block_plan_refused_by_order_entry_points():
    import ctypes

    L = sht.lib()
    P = sht.GJPlan(64, 64, 0, leaf_cols=16, host_only=True)
    x = np.zeros(4)
    assert L.sht_legendre_synthesize(P.handle, 0, x.ctypes.data, x.ctypes.data, None) == 6  # SHT_ERR_UNSUPPORTED
    assert L.sht_plan_nodes(P.handle, x.ctypes.data, x.ctypes.data) == 6
    assert L.sht_plan_save(P.handle, b"/nonexistent/x") == 6
    Q = sht.Plan(8, 1e-12, host_only=True)
    assert L.sht_gj_forward(Q.handle, 0, x.ctypes.data, x.ctypes.data, None) == 6
    c = ctypes.c_int()
    assert L.sht_gj_launches(Q.handle, 0, 0, ctypes.byref(c)) == 6
    out = ctypes.c_void_p()
    assert L.sht_gj_plan_create(0, 0, 0, 1e-12, None, ctypes.byref(out)) == 1
    assert L.sht_gj_plan_create(10, 0, 2, 1e-12, None, ctypes.byref(out)) == 1
    assert L.sht_gj_plan_create(sht_max_n() + 1, 0, 0, 1e-12, None, ctypes.byref(out)) == 1
    P.close()
    Q.close()


def sht_max_n():
    return 40000  # SHT_GJ_MAX_N
