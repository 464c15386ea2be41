"""Refusals of the C ABI that happen on the host before any device work, so
they are checked without a GPU: NULL or misaligned arguments, unknown
precisions, an out-of-range static scratch slot, and plans built with
host_only (which own no device memory) passed to entry points that launch.
Addresses below are never dereferenced: each call is refused first."""

import ctypes

import pytest

from paper_0910_5435_gb300 import sht

INVALID, UNSUPPORTED = 1, 6
A, B, C = 1 << 20, 2 << 20, 3 << 20  # 16-byte aligned stand-in addresses


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return sht.lib()


@pytest.fixture(scope="module")
def plan(lib):
    P = sht.Plan(8, 1e-12, leaf_cols=4, host_only=True)
    yield P.handle
    P.close()


def test_launching_entry_points_refuse_host_only_plans(lib, plan):
    for prec in (0, 1, 2, 3):
        assert lib.sht_legendre_synthesize(plan, prec, A, B, None) == UNSUPPORTED
        assert lib.sht_legendre_analyze(plan, prec, A, B, None) == UNSUPPORTED
        assert lib.sht_legendre_synthesize_adjoint(plan, prec, A, B, None) == UNSUPPORTED
        assert lib.sht_phi_synthesize(plan, prec, A, B, C, None) == UNSUPPORTED
        assert lib.sht_phi_analyze(plan, prec, A, B, None) == UNSUPPORTED
        assert lib.sht_synthesize(plan, prec, A, B, C, None) == UNSUPPORTED
        assert lib.sht_analyze(plan, prec, A, B, C, None) == UNSUPPORTED
        assert lib.sht_legendre_synthesize_noalloc(plan, prec, A, B, 0, None, None) == UNSUPPORTED
    assert lib.sht_direct_prepare(plan) == UNSUPPORTED
    assert lib.sht_direct_synthesize(plan, A, B, None) == UNSUPPORTED
    assert lib.sht_direct_analyze(plan, A, B, None) == UNSUPPORTED
    assert lib.sht_last_device_status(plan, None) == UNSUPPORTED
    assert lib.sht_trace_enable(plan, 1) == UNSUPPORTED
    buf = (ctypes.c_ulonglong * 64)()
    assert lib.sht_trace_read(plan, buf, 0) == UNSUPPORTED


def test_unknown_precision_and_null_buffers(lib, plan):
    for bad in (-1, 4, 99):
        assert lib.sht_legendre_synthesize(plan, bad, A, B, None) == INVALID
        assert lib.sht_legendre_analyze(plan, bad, A, B, None) == INVALID
        assert lib.sht_phi_synthesize(plan, bad, A, B, C, None) == INVALID
        assert lib.sht_synthesize(plan, bad, A, B, C, None) == INVALID
        assert lib.sht_prepare(plan, bad) == INVALID
    assert lib.sht_legendre_synthesize(plan, 0, None, B, None) == INVALID
    assert lib.sht_legendre_analyze(plan, 0, A, None, None) == INVALID
    assert lib.sht_phi_analyze(plan, 0, None, B, None) == INVALID
    assert lib.sht_plan_nodes(plan, None, None) == INVALID
    size = ctypes.c_size_t(0)
    assert lib.sht_plan_stream(plan, 0, 2, None, ctypes.byref(size), None) == INVALID
    assert lib.sht_plan_stream(plan, 7, 0, None, ctypes.byref(size), None) == INVALID


def test_static_scratch_slot_and_status_word_checked_first(lib, plan):
    for slot in (-1, sht.NOALLOC_MAX_SLOTS, 1 << 30):
        assert lib.sht_legendre_synthesize_noalloc(plan, 0, A, B, slot, None, None) == INVALID
        assert str(sht.NOALLOC_MAX_SLOTS).encode() in lib.sht_last_error_detail()
    assert lib.sht_legendre_synthesize_noalloc(plan, 0, A, B, 0, A + 2, None) == INVALID  # misaligned status


def test_batches_refuse_bad_arguments_and_host_only_plans(lib, plan):
    out = ctypes.c_void_p(123)
    plans = (ctypes.c_void_p * 2)(plan, plan)
    assert lib.sht_batch_create(2, plans, 0, ctypes.byref(out)) == UNSUPPORTED and not out.value
    assert lib.sht_batch_create(0, plans, 0, ctypes.byref(out)) == INVALID and not out.value
    assert lib.sht_batch_create(2, plans, 9, ctypes.byref(out)) == INVALID
    assert lib.sht_batch_create(2, None, 0, ctypes.byref(out)) == INVALID
    with_null = (ctypes.c_void_p * 2)(plan, None)
    assert lib.sht_batch_create(2, with_null, 0, ctypes.byref(out)) == INVALID
    assert lib.sht_batch_create(2, plans, 0, None) == INVALID
    for call in (lib.sht_batch_synthesize, lib.sht_batch_analyze, lib.sht_batch_synthesize_adjoint):
        assert call(None, A, B, None) == INVALID
    assert lib.sht_batch_synthesize_grid(None, A, B, C, None) == INVALID
    assert lib.sht_batch_analyze_grid(None, A, B, C, None) == INVALID
    assert lib.sht_batch_last_device_status(None, None) == INVALID
    assert lib.sht_batch_autotune(None, 0, A, B, 1, None) == INVALID
    assert lib.sht_batch_get_config(None, 0, None, None, None, None) == INVALID
    assert lib.sht_batch_destroy(None) == 0


def test_workspace_size_of_a_host_only_plan(lib, plan):
    assert lib.sht_workspace_bytes(plan, 0) == 16 * 16 * 16
    assert lib.sht_workspace_bytes(plan, 1) == 16 * 16 * 8
    assert lib.sht_workspace_bytes(None, 0) == 0
