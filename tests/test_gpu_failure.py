"""Failure detection on the GPU without a fault: a plan whose stream plants
one op that waits for its own completion (a flag nothing sets).  The sweep's
bounded wait gives up (about 2 s), every warp of the CTA returns, copies in
flight are drained, and the host reads SHT_ERR_TIMEOUT from the device
status word; the context stays usable and the next launches are correct."""

import time

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht as _sht
    assert torch.cuda.is_available()
    return _sht


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_unmet_dependency_times_out_and_context_survives(sht):
    l = 16
    bad = sht.Plan(l, 1e-12, leaf_cols=4, debug_unmet_dependency=1)
    good = sht.Plan(l, 1e-12, leaf_cols=4)
    beta = torch.from_numpy(inputs.random_beta(l, seed=21)).cuda()
    G = torch.zeros((2 * l, 2 * l), dtype=torch.complex128, device="cuda")
    for _ in range(2):  # twice: the queue counter is reset after a timeout
        t0 = time.perf_counter()
        sht.sht_legendre_synthesize(bad, 0, beta, G)
        torch.cuda.synchronize()
        assert sht.sht_last_device_status(bad) == 5  # SHT_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 30
    # same process, same context: a correct plan still gives correct results
    sht.sht_legendre_synthesize(good, 0, beta, G)
    torch.cuda.synchronize()
    assert sht.sht_last_device_status(good) == 0
    assert rel(G.cpu().numpy(), oracle.legendre_synthesis(beta.cpu().numpy(), l)) < 1e-10
    # and the analysis stream of the planted plan fails the same way
    b = torch.zeros_like(beta)
    sht.sht_legendre_analyze(bad, 0, G, b)
    torch.cuda.synchronize()
    assert sht.sht_last_device_status(bad) == 5
