"""GPU parity of the paper's own matrices (Section 4, eqs. transform and
transform2) against the oracle's direct products (oracle/gauss_jacobi.py).

A single-block plan (sht_gj_plan_create) factors the n x n matrix of order
m on the host and applies it on the GPU level by level (one sweep launch per
butterfly level, vectors in global memory).  Inputs: two unit-norm
U(-1, 1) real vectors per call, as the real and imaginary parts (the
paper's test vectors, Section 5).  Checked per precision: the forward
transform against A beta (relative l2 and the paper's eps_fwd, the largest
entry difference), the inverse against A^T alpha, and eps_inv (forward then
inverse, against the input).  Tolerances: float64 at eps_id = 1e-12 1e-10,
split float32 1e-9, float32 2e-5 (relative l2); eps_fwd and eps_inv within
the same bounds, as the vectors have unit norm.
"""

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 2: 1e-9, 3: 1e-9, 1: 2e-5}
CDT = {0: torch.complex128, 2: torch.complex128, 3: torch.complex128, 1: torch.complex64}


@pytest.fixture(scope="module")
def sht():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht as _sht
    assert torch.cuda.is_available()
    return _sht


def unit_vectors(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1, 1, (n, 2))
    v /= np.linalg.norm(v, axis=0)
    return v[:, 0] + 1j * v[:, 1]


def run(sht, P, prec, x, inverse=False):
    xin = torch.from_numpy(np.asarray(x)).to(CDT[prec]).cuda()
    y = torch.full_like(xin, float("nan"))
    (sht.sht_gj_inverse if inverse else sht.sht_gj_forward)(P, prec, xin, y)
    torch.cuda.synchronize()
    assert sht.sht_last_device_status(P) == 0
    return y.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,m,p", [(300, 300, 0), (300, 300, 1), (257, 0, 0), (1250, 1250, 0), (1250, 1250, 1),
                                   (1250, 0, 1)])
def test_forward_inverse_match_oracle(sht, n, m, p):
    P = sht.GJPlan(n, m, p, eps_id=1e-12, leaf_cols=32)
    A = oracle.gj_matrix(m, p, n)
    beta = unit_vectors(n, 11 + p)
    alpha_o = A @ beta
    alpha_in = unit_vectors(n, 21 + p)
    beta_o = A.T @ alpha_in
    for prec in (0, 2, 3, 1):
        P.prepare(prec)
        a = run(sht, P, prec, beta)
        assert rel(a, alpha_o) < TOL[prec], (prec, rel(a, alpha_o))
        assert np.max(np.abs(a - alpha_o)) < TOL[prec]  # eps_fwd
        b = run(sht, P, prec, alpha_in, inverse=True)
        assert rel(b, beta_o) < TOL[prec], (prec, rel(b, beta_o))
        back = run(sht, P, prec, a, inverse=True)
        assert np.max(np.abs(back - beta)) < 2 * TOL[prec]  # eps_inv
    assert P.launches(0, 0) >= 3 and P.launches(0, 1) >= 3
    P.close()


def test_m_equals_n_2500_sampled_rows(sht):
    """n = m = 2500 (Table evens' second size): rows i of A beta on a stride,
    from the oracle row by row."""
    n = m = 2500
    P = sht.GJPlan(n, m, 0, eps_id=1e-12, leaf_cols=60)
    beta = unit_vectors(n, 31)
    rows = list(range(0, n, 97)) + [n - 1]
    ref = oracle.gj_forward(beta, m, 0, rows=rows)
    for prec in (0, 2):
        a = run(sht, P, prec, beta)
        assert rel(a[rows], ref) < TOL[prec]
        back = run(sht, P, prec, a, inverse=True)
        assert np.max(np.abs(back - beta)) < 2 * TOL[prec]
    P.close()


def test_in_place_and_repeated_calls(sht):
    n, m = 300, 300
    P = sht.GJPlan(n, m, 1, eps_id=1e-12, leaf_cols=32)
    beta = unit_vectors(n, 41)
    first = run(sht, P, 0, beta)
    x = torch.from_numpy(beta).cuda()
    for _ in range(3):
        sht.sht_gj_forward(P, 0, x, x)  # in place
        sht.sht_gj_inverse(P, 0, x, x)
    torch.cuda.synchronize()
    assert np.max(np.abs(x.cpu().numpy() - beta)) < 1e-10
    assert np.array_equal(run(sht, P, 0, beta), first)  # deterministic
    P.close()


def test_order_entry_points_refuse_single_block_plans(sht):
    P = sht.GJPlan(64, 64, 0, leaf_cols=16)
    b = torch.zeros(64 * 129, dtype=torch.complex128, device="cuda")
    G = torch.zeros((128, 128), dtype=torch.complex128, device="cuda")
    with pytest.raises(sht.ShtError) as e:
        sht.sht_legendre_synthesize(P, 0, b, G)
    assert e.value.code == 6  # SHT_ERR_UNSUPPORTED
    Q = sht.Plan(16, 1e-12, leaf_cols=8)
    x = torch.zeros(16, dtype=torch.complex128, device="cuda")
    with pytest.raises(sht.ShtError) as e:
        sht.sht_gj_forward(Q, 0, x, x)
    assert e.value.code == 6
    P.close()
    Q.close()
