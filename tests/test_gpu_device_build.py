"""Factorizations built on the GPU (sht_plan_opts.device_build = 1).

The device builder generates the same columns as the host builder (same
recurrence, same rounding of each product and sum) and runs the same
column-pivoted QR and depth-first merges (Section 3), so its plans must
  * transform like the host's: parity against the float64 oracle at the
    usual tolerances, for every precision and both directions;
  * keep the same rows after trimming and nearly the same ranks (the QR's
    reductions round in another order, which can move a residual norm
    across eps_id);
  * be reproducible: two device builds give identical streams.
The streams are also checked on the host alone (tests/stream_emulator.py),
which separates the builder from the sweep kernel.
"""

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import inputs
from tests.stream_emulator import emulate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 2: 1e-9, 3: 1e-9, 1: 2e-5}
NDT = {0: np.complex128, 2: np.complex128, 3: np.complex128, 1: np.complex64}
CDT = {0: torch.complex128, 2: torch.complex128, 3: torch.complex128, 1: torch.complex64}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sht():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht as _sht
    assert torch.cuda.is_available()
    return _sht


def synth(sht, P, prec, beta):
    l = P.l
    b = torch.from_numpy(beta.astype(NDT[prec])).cuda()
    G = torch.full((2 * l, 2 * l), float("nan"), dtype=CDT[prec], device="cuda")
    sht.sht_legendre_synthesize(P, prec, b, G)
    torch.cuda.synchronize()
    assert sht.sht_last_device_status(P) == 0
    return G.cpu().numpy()


def analysis(sht, P, prec, G):
    l = P.l
    g = torch.from_numpy(G.astype(NDT[prec])).cuda()
    b = torch.full((inputs.triangle_size(l),), float("nan"), dtype=CDT[prec], device="cuda")
    sht.sht_legendre_analyze(P, prec, g, b)
    torch.cuda.synchronize()
    assert sht.sht_last_device_status(P) == 0
    return b.cpu().numpy()


@pytest.mark.parametrize("l,C", [(1, 4), (2, 4), (16, 4), (64, 16), (128, 16), (128, 64)])
def test_device_built_plan_matches_oracle(sht, l, C):
    P = sht.Plan(l, 1e-12, leaf_cols=C, device_build=True)
    beta = inputs.random_beta(l, seed=11)
    Gin = inputs.random_G(l, seed=12)
    Go = oracle.legendre_synthesis(beta, l)
    bo = oracle.legendre_analysis(Gin, l)
    for prec in (0, 2, 3, 1):
        P.prepare(prec)
        assert rel(synth(sht, P, prec, beta), Go) < TOL[prec], prec
        assert rel(analysis(sht, P, prec, Gin), bo) < TOL[prec], prec
    P.close()


@pytest.mark.parametrize("l,C", [(64, 16), (256, 32)])
def test_device_streams_on_the_host_emulator(sht, l, C):
    """The device-built float64 streams, applied by the host emulator, agree
    with the oracle: the builder is right independently of the kernel."""
    P = sht.Plan(l, 1e-12, leaf_cols=C, device_build=True)
    beta = inputs.random_beta(l, seed=13)
    Ge = emulate(P.stream(0, 0), P.page_bytes, l, 0, 0, beta)
    ms = list(range(0, 2 * l, 7))
    Go = oracle.legendre_synthesis(beta, l, orders=ms)
    assert rel(Ge[ms], Go[ms]) < 1e-10
    Gin = inputs.random_G(l, seed=14)
    be = emulate(P.stream(0, 1), P.page_bytes, l, 0, 1, Gin)
    off = oracle.triangle_offsets(l)
    sel = np.concatenate([np.arange(off[m], off[m + 1]) for m in ms])
    bo = oracle.legendre_analysis(Gin, l, orders=ms)
    assert rel(be[sel], bo[sel]) < 1e-10
    P.close()


@pytest.mark.parametrize("l,C", [(128, 16), (256, 32)])
def test_device_and_host_builds_agree(sht, l, C):
    Pd = sht.Plan(l, 1e-12, leaf_cols=C, device_build=True)
    Ph = sht.Plan(l, 1e-12, leaf_cols=C)
    sd, sh = Pd.stats(), Ph.stats()
    # identical columns: identical trimming, units and levels
    for key in ("rows_kept", "rows_total", "dense_values", "max_levels", "n_units"):
        assert sd[key] == sh[key], key
    # the ranks move by rounding only
    assert abs(sd["n_blocks"] - sh["n_blocks"]) <= 0.01 * sh["n_blocks"]
    assert abs(sd["k_avg"] - sh["k_avg"]) <= 0.005 * sh["k_avg"]
    assert abs(sd["k_max"] - sh["k_max"]) <= 1
    assert abs(sd["factor_values"] - sh["factor_values"]) <= 0.01 * sh["factor_values"]
    # the peak memory of the depth-first order, replayed from the device's ranks
    assert abs(sd["m_max_words"] - sh["m_max_words"]) <= 0.02 * sh["m_max_words"]
    # both builders end with the strong rank-revealing step: coefficients <= 2
    assert sd["max_abs_T"] <= 2.0 + 1e-12 and sh["max_abs_T"] <= 2.0 + 1e-12
    # the two transforms agree to the ID precision
    beta = inputs.random_beta(l, seed=15, decay=True)
    assert rel(synth(sht, Pd, 0, beta), synth(sht, Ph, 0, beta)) < 1e-10
    Pd.close()
    Ph.close()


def test_device_build_is_reproducible(sht):
    a = sht.Plan(128, 1e-12, leaf_cols=16, device_build=True)
    b = sht.Plan(128, 1e-12, leaf_cols=16, device_build=True)
    def same(q, d):
        # (page region, value region) of each plan's stream
        return all(np.array_equal(x, y) for x, y in zip(a.stream(q, d), b.stream(q, d)))

    assert same(0, 0) and same(0, 1)
    a.prepare(1)
    b.prepare(1)
    assert same(1, 0)
    a.close()
    b.close()


def test_small_arena_builds_in_waves(sht):
    """A 1 MB record arena cannot hold a whole l = 128 build: the device
    builds the blocks that fit, then the rest in further launches (one CTA at
    a time when a launch finished nothing), and the streams are those of a
    build in one launch."""
    a = sht.Plan(128, 1e-12, leaf_cols=16, device_build=True)
    b = sht.Plan(128, 1e-12, leaf_cols=16, device_build=True, device_build_arena_mb=1)
    for d in (0, 1):
        assert all(np.array_equal(x, y) for x, y in zip(a.stream(0, d), b.stream(0, d)))
    beta = inputs.random_beta(128, seed=16)
    assert rel(synth(sht, b, 0, beta), oracle.legendre_synthesis(beta, 128)) < 1e-10
    a.close()
    b.close()


def test_arena_too_small_for_one_block_is_an_error(sht):
    with pytest.raises(sht.ShtError) as e:
        sht.Plan(1024, 1e-12, leaf_cols=32, device_build=True, device_build_arena_mb=1)
    assert e.value.code == 1
    assert b"cannot hold one unit" in sht.lib().sht_last_error_detail()


def test_device_build_l1024_sampled_orders(sht):
    """The bench configuration (l = 1024, C = 32, 8 KB pages) built on the
    device, checked on sampled orders against the oracle."""
    l = 1024
    P = sht.Plan(l, 1e-12, leaf_cols=32, device_build=True)
    beta = inputs.random_beta(l, seed=3, decay=True)
    ms = [0, 1, 2, 511, 1024, 1025, 2046, 2047]
    Go = oracle.legendre_synthesis(beta, l, orders=ms)
    G = synth(sht, P, 0, beta)
    assert rel(G[ms], Go[ms]) < 1e-10
    Gin = inputs.random_G(l, seed=4)
    bo = oracle.legendre_analysis(Gin, l, orders=ms)
    off = oracle.triangle_offsets(l)
    sel = np.concatenate([np.arange(off[m], off[m + 1]) for m in ms])
    b = analysis(sht, P, 0, Gin)
    assert rel(b[sel], bo[sel]) < 1e-10
    P.close()
