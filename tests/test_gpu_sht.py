"""GPU parity of the phi stage (cuFFT, length 4l-1) and of the full SHT
(butterfly Legendre stage + phi stage) against the float64 oracle's naive
DFT and direct transform (Section 2, eqs. expansion, alternate_expansion,
phis).  All calls go through the C ABI."""

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 2: 1e-9, 3: 1e-9, 1: 2e-5}
CDT = {0: torch.complex128, 2: torch.complex128, 3: torch.complex128, 1: torch.complex64}
RDT = {0: torch.float64, 2: torch.float64, 3: torch.float64, 1: torch.float32}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sht():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht as _sht
    return _sht


_plans = {}


def plan(sht, l, C=16):
    if (l, C) not in _plans:
        _plans[(l, C)] = sht.Plan(l, 1e-12, leaf_cols=C)
    return _plans[(l, C)]


def workspace(sht, P, prec):
    n = sht.sht_workspace_bytes(P, prec)
    return torch.empty(n // 16 + 1, dtype=torch.complex128, device="cuda")


@pytest.mark.parametrize("l", [1, 3, 16, 64])
@pytest.mark.parametrize("prec", [0, 1])
def test_phi_stage_matches_naive_dft(sht, l, prec):
    P = plan(sht, l)
    G = inputs.random_G(l, seed=l)
    G[0] = G[0].real  # real field: G^0 is real
    g = torch.from_numpy(G).to(CDT[prec]).cuda()
    f = torch.empty((2 * l, 4 * l - 1), dtype=RDT[prec], device="cuda")
    sht.sht_phi_synthesize(P, prec, g, f, workspace(sht, P, prec))
    torch.cuda.synchronize()
    fo = oracle.phi_synthesis(G, l)
    assert rel(f.cpu().numpy(), fo) < TOL[prec]
    g2 = torch.empty_like(g)
    sht.sht_phi_analyze(P, prec, f, g2)
    torch.cuda.synchronize()
    assert rel(g2.cpu().numpy(), oracle.phi_analysis(fo, l)) < TOL[prec]


@pytest.mark.parametrize("l,C", [(2, 4), (16, 4), (64, 16), (128, 16)])
@pytest.mark.parametrize("prec", [0, 2, 3, 1])
def test_full_sht_matches_oracle(sht, l, C, prec):
    P = plan(sht, l, C)
    beta = inputs.random_beta(l, seed=300 + l)
    b = torch.from_numpy(beta).to(CDT[prec]).cuda()
    f = torch.empty((2 * l, 4 * l - 1), dtype=RDT[prec], device="cuda")
    ws = workspace(sht, P, prec)
    sht.sht_synthesize(P, prec, b, f, ws)
    torch.cuda.synchronize()
    assert sht.sht_last_device_status(P) == 0
    fo = oracle.sht_synthesis(beta, l)
    assert rel(f.cpu().numpy(), fo) < TOL[prec]
    grid = inputs.random_grid(l, seed=400 + l)
    g = torch.from_numpy(grid).to(RDT[prec]).cuda()
    bb = torch.empty_like(b)
    sht.sht_analyze(P, prec, g, bb, ws)
    torch.cuda.synchronize()
    assert rel(bb.cpu().numpy(), oracle.sht_analysis(grid, l)) < TOL[prec]


def test_full_round_trip_l512(sht):
    l = 512
    P = plan(sht, l, 64)
    beta = inputs.random_beta(l, seed=12, decay=True)
    b = torch.from_numpy(beta).cuda()
    f = torch.empty((2 * l, 4 * l - 1), dtype=torch.float64, device="cuda")
    ws = workspace(sht, P, 0)
    sht.sht_synthesize(P, 0, b, f, ws)
    back = torch.empty_like(b)
    sht.sht_analyze(P, 0, f, back, ws)
    torch.cuda.synchronize()
    assert rel(back.cpu().numpy(), beta) < 1e-10


def test_special_fields(sht):
    """f = 1 <-> beta^0_0 = sqrt 2 and f = cos(theta) <-> beta^0_1 = sqrt(2/3)
    (Section 2.3, eq. association: P-bar^0_0 = 1/sqrt 2, P-bar^0_1 = sqrt(3/2) x)."""
    l = 8
    P = plan(sht, l, 4)
    x, _ = P.nodes()
    ws = workspace(sht, P, 0)
    b = torch.empty(inputs.triangle_size(l), dtype=torch.complex128, device="cuda")
    for field, k, val in [(np.ones((2 * l, 4 * l - 1)), 0, np.sqrt(2)),
                          (np.repeat(x[:, None], 4 * l - 1, axis=1), 1, np.sqrt(2 / 3))]:
        sht.sht_analyze(P, 0, torch.from_numpy(field).cuda(), b, ws)
        torch.cuda.synchronize()
        ref = np.zeros(inputs.triangle_size(l), dtype=complex)
        ref[k] = val
        assert np.max(np.abs(b.cpu().numpy() - ref)) < 1e-13
