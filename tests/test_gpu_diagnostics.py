"""sht_measure_fp64_fma: the float64 FMA loop the float64 kernels are
compared with lands within a plausible band of the rate derived from unit
counts and clocks (2 DFMA per clock per SM on this part); sht_measure_fp64_mma:
the float64 tensor-core loop beside it."""

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_plausible():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = 2 * sms * 2.07e9 * 2 / 1e12  # TFLOP/s at the maximum clock
    t = sht.measure_fp64_fma()
    assert 0.3 * derived < t < 1.2 * derived, (t, derived)


def test_fp64_mma_rate_is_positive_and_bounded():
    """sht_measure_fp64_mma: the float64 warp-MMA loop finishes, reports a
    positive rate, and stays below the dense float64 tensor figure of the
    parts that have one (tens of TFLOP/s)."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht
    t = sht.measure_fp64_mma()
    assert 0.0 < t < 100.0, t
