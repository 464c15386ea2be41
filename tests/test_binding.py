"""Host-side checks of the Python binding that need no GPU: a batch whose
plan was closed, or which was closed itself, refuses every launch before
the library is called."""

import types

import pytest

from paper_0910_5435_gb300 import sht


class _StandInBatch(sht.Batch):
    def close(self):  # its handle is not the library's: nothing to destroy
        self.handle = None


def _batch(handle, plan_handles):
    b = object.__new__(_StandInBatch)  # no device: the fields a launch checks
    b.handle = handle
    b.plans = [types.SimpleNamespace(handle=h) for h in plan_handles]
    b.prec = sht.SHT_FP64
    return b


@pytest.mark.parametrize("call", [
    lambda b: sht.sht_batch_synthesize(b, 0, 0, stream=0),
    lambda b: sht.sht_batch_analyze(b, 0, 0, stream=0),
    lambda b: sht.sht_batch_synthesize_adjoint(b, 0, 0, stream=0),
    lambda b: sht.sht_batch_synthesize_grid(b, [], [], [], stream=0),
    lambda b: sht.sht_batch_analyze_grid(b, [], [], [], stream=0),
    lambda b: sht.sht_batch_autotune(b, 0, 0, 0, stream=0),
])
def test_launches_refused_after_a_plan_or_the_batch_is_closed(call):
    with pytest.raises(sht.ShtError) as e:
        call(_batch(1234, [5678, None]))
    assert e.value.code == 1 and "plan of this batch was closed" in str(e.value)
    with pytest.raises(sht.ShtError) as e:
        call(_batch(None, [5678]))
    assert e.value.code == 1 and "batch is closed" in str(e.value)


def test_closing_a_plan_closes_its_cached_batches():
    closed = []
    P = object.__new__(sht.Plan)
    P.handle = None  # nothing to destroy in the library
    P._autograd_batches = {(0, 16): types.SimpleNamespace(close=lambda: closed.append(1))}
    P.close()
    assert closed == [1] and "_autograd_batches" not in P.__dict__
