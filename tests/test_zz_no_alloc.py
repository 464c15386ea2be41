"""The allocation-free Legendre synthesis (sht_legendre_synthesize_noalloc)
against sht_legendre_synthesize, through the C ABI.

Tolerances (relative l2, complex as 2 reals) are those of the parity tests:
float64 1e-10, split float32 1e-9, float32 2e-5.  Both entry points run the
same kernel on the same streams, so they agree far inside these.
"""

import numpy as np
import pytest

from paper_0910_5435_gb300 import inputs

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


def rel(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("prec", [0, 2, 3, 1])
def test_two_calls_match_the_allocating_entry_point(sht, prec):
    l = 128
    P = sht.Plan(l, 1e-12, leaf_cols=16)
    P.prepare(prec)
    beta = torch.from_numpy(inputs.random_beta(l, seed=41)).to(CDT[prec]).cuda()
    ref = torch.full((2 * l, 2 * l), float("nan"), dtype=CDT[prec], device="cuda")
    sht.sht_legendre_synthesize(P, prec, beta, ref)
    torch.cuda.synchronize()
    assert sht.sht_last_device_status(P) == 0
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")  # must be zeroed by the call
    for _ in range(2):
        G = torch.full_like(ref, float("nan"))
        sht.sht_legendre_synthesize_noalloc(P, prec, beta, G, slot=3, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert not torch.isnan(torch.view_as_real(G)).any()
        assert rel(G, ref) < TOL[prec]
    P.close()


def test_slots_without_status_word(sht):
    """Different slots and no status word give the same result."""
    l = 64
    P = sht.Plan(l, 1e-12, leaf_cols=16)
    beta = torch.from_numpy(inputs.random_beta(l, seed=42)).cuda()
    ref = torch.empty((2 * l, 2 * l), dtype=torch.complex128, device="cuda")
    sht.sht_legendre_synthesize(P, 0, beta, ref)
    for slot in (0, sht.NOALLOC_MAX_SLOTS - 1):
        G = torch.full_like(ref, float("nan"))
        sht.sht_legendre_synthesize_noalloc(P, 0, beta, G, slot=slot)
        torch.cuda.synchronize()
        assert rel(G, ref) < TOL[0]
    P.close()


def test_rejections(sht):
    """A slot beyond the static array and a precision not yet on the device
    are refused before any launch."""
    l = 32
    P = sht.Plan(l, 1e-12, leaf_cols=8)
    beta = torch.from_numpy(inputs.random_beta(l, seed=43)).cuda()
    G = torch.empty((2 * l, 2 * l), dtype=torch.complex128, device="cuda")
    for slot in (-1, sht.NOALLOC_MAX_SLOTS):
        with pytest.raises(sht.ShtError) as e:
            sht.sht_legendre_synthesize_noalloc(P, 0, beta, G, slot=slot)
        assert e.value.code == 1
        assert str(sht.NOALLOC_MAX_SLOTS).encode() in sht.lib().sht_last_error_detail()
    with pytest.raises(sht.ShtError) as e:
        sht.sht_legendre_synthesize_noalloc(P, 1, beta.to(torch.complex64), G.to(torch.complex64))
    assert e.value.code == 6
    P.close()


def test_device_and_pending_error_untouched_and_nothing_allocated(sht):
    """The call leaves the caller's current device current, and ten calls
    change neither the device's free memory nor the torch allocator's."""
    l = 64
    P = sht.Plan(l, 1e-12, leaf_cols=16)
    beta = torch.from_numpy(inputs.random_beta(l, seed=44)).cuda()
    G = torch.empty((2 * l, 2 * l), dtype=torch.complex128, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sht.sht_legendre_synthesize_noalloc(P, 0, beta, G, slot=5, status=status)  # first call: set-up
    torch.cuda.synchronize()
    dev = torch.cuda.current_device()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(10):
        sht.sht_legendre_synthesize_noalloc(P, 0, beta, G, slot=5, status=status)
        assert torch.cuda.current_device() == dev
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    if torch.cuda.device_count() > 1:
        # a plan of device 0 called while another device is current
        with torch.cuda.device(1):
            sht.sht_legendre_synthesize_noalloc(P, 0, beta, G, slot=6)
            assert torch.cuda.current_device() == 1
        torch.cuda.synchronize(0)
    P.close()


def test_timeout_is_reported_in_the_status_word_and_the_slot_recovers(sht):
    """A plan whose first op waits for a completion that never comes (the
    failure-detection option of the plan): each call's bounded wait gives up
    (about 2 s) and writes SHT_ERR_TIMEOUT into the caller's status word; the
    next call on the same slot with a sound plan clears the slot's dirty
    counter and matches the oracle."""
    import oracle

    l = 32
    bad = sht.Plan(l, 1e-12, leaf_cols=8, debug_unmet_dependency=1)
    good = sht.Plan(l, 1e-12, leaf_cols=8)
    beta_np = inputs.random_beta(l, seed=45)
    beta = torch.from_numpy(beta_np).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        G = torch.empty((2 * l, 2 * l), dtype=torch.complex128, device="cuda")
        sht.sht_legendre_synthesize_noalloc(bad, 0, beta, G, slot=7, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 5
    G = torch.full((2 * l, 2 * l), float("nan"), dtype=torch.complex128, device="cuda")
    sht.sht_legendre_synthesize_noalloc(good, 0, beta, G, slot=7, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = oracle.legendre_synthesis(beta_np, l)
    assert np.linalg.norm(G.cpu().numpy() - ref) / np.linalg.norm(ref) < TOL[0]
    bad.close()
    good.close()
