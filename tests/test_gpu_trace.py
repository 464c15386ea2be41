"""The sweep's per-op trace (sht_trace_enable / sht_trace_read): the counters
count exactly the ops and work items of the plan's streams, the cycle
counters are filled, and tracing leaves the results unchanged bit for bit."""

import numpy as np
import pytest

from paper_0910_5435_gb300 import inputs
from tests import stream_emulator as se

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONSUMER_WARPS = 16  # the plan default: every warp of a CTA walks each item


@pytest.fixture(scope="module")
def sht():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht as _sht
    assert torch.cuda.is_available()
    return _sht


def stream_counts(plan, prec, direction):
    records, values = plan.stream(prec, direction)
    chunk = plan.page_bytes
    items = sum(1 for _ in se.iter_items(records, chunk))
    compute = control = 0
    for h, _, _ in se.iter_ops((records, values), chunk):
        if se.OP_SYN <= int(h["kind"]) <= se.OP_ANA:
            compute += 1
        else:
            control += 1
    return items, compute, control


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_trace_counts_every_op_and_item_and_changes_nothing(sht, prec):
    l = 96
    P = sht.Plan(l, 1e-12, leaf_cols=16)
    P.prepare(prec)
    cdt = torch.complex64 if prec == 1 else torch.complex128
    beta = torch.from_numpy(inputs.random_beta(l, seed=5)).to(cdt).cuda()
    G0 = torch.empty((2 * l, 2 * l), dtype=cdt, device="cuda")
    G1 = torch.empty_like(G0)
    b0 = torch.empty_like(beta)
    b1 = torch.empty_like(beta)
    sht.sht_legendre_synthesize(P, prec, beta, G0)
    sht.sht_legendre_analyze(P, prec, G0, b0)
    torch.cuda.synchronize()
    sht.sht_trace_enable(P, True)
    try:
        for direction in (0, 1):
            sht.sht_trace_read(P, reset=True)
            if direction == 0:
                sht.sht_legendre_synthesize(P, prec, beta, G1)
            else:
                sht.sht_legendre_analyze(P, prec, G0, b1)
            torch.cuda.synchronize()
            t = sht.sht_trace_read(P, reset=True)
            items, compute, control = stream_counts(P, prec, direction)
            assert t["n_gemv"] == compute
            assert t["n_control"] == control
            assert t["n_items"] == items * CONSUMER_WARPS
            assert t["exec_gemv"] > 0 and t["complete"] >= 0
            # read with reset: the counters start again from zero
            assert all(v == 0 for v in sht.sht_trace_read(P, reset=False).values())
    finally:
        sht.sht_trace_enable(P, False)
    assert sht.sht_last_device_status(P) == 0
    assert torch.equal(G0, G1)
    assert torch.equal(b0, b1)
