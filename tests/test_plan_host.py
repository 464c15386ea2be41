"""Host-side checks of the product's precomputation (no GPU): the library is
driven through its C ABI with host-only plans, and its factor streams are
decoded and applied by tests/stream_emulator.py, then compared with the oracle.
"""

import math

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import inputs, sht
from tests.stream_emulator import check_races, emulate, iter_ops



def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("l", [1, 2, 8, 64, 300])
def test_nodes_match_oracle(l):
    """The product's Gauss-Legendre nodes (Section 2, eq. thetas), computed by
    its own code, agree with the oracle's to a few ulp (weights: the n-scaled
    roundoff of the degree recurrence near the poles)."""
    P = sht.Plan(l, 1e-12, host_only=True)
    x, w = P.nodes()
    xo, wo = oracle.gl_nodes_weights(2 * l)
    assert np.max(np.abs(x - xo)) < 4e-16
    assert np.max(np.abs(w / wo - 1)) < 4e-15 * 2 * l


@pytest.mark.parametrize("l,C", [(1, 4), (4, 2), (16, 4), (64, 16), (64, 64), (128, 16)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-10), (1, 2e-5)])
def test_streams_reproduce_oracle(l, C, prec, tol):
    """Synthesis, analysis and the adjoint, applied from the decoded factor
    streams, match the direct oracle transform (Section 2) within the stated
    tolerance of each precision (rel. l2; float64 factors at eps_id = 1e-12)."""
    P = sht.Plan(l, 1e-12, leaf_cols=C, host_only=True)
    beta = inputs.random_beta(l, seed=l + C)
    Go = oracle.legendre_synthesis(beta, l)
    G = emulate(P.stream(prec, 0), P.page_bytes, l, prec, 0, beta)
    assert rel(G, Go) < tol
    Gin = inputs.random_G(l, seed=7)
    bo = oracle.legendre_analysis(Gin, l)
    b = emulate(P.stream(prec, 1), P.page_bytes, l, prec, 1, Gin)
    assert rel(b, bo) < tol
    _, w = P.nodes()
    ba = emulate(P.stream(prec, 1), P.page_bytes, l, prec, 1, Gin, prescale=1.0 / w[l:])
    assert rel(ba, oracle.legendre_adjoint(Gin, l)) < tol


def test_butterfly_levels_are_exercised():
    """l = 128 with C = 16 must build multi-level butterflies (Section 2.2,
    Figure multi) and compress the operator."""
    P = sht.Plan(128, 1e-12, leaf_cols=16, host_only=True)
    s = P.stats()
    assert s["max_levels"] >= 3
    assert s["n_blocks"] > 100
    assert s["factor_values"] < s["dense_values"]
    assert 0 < s["k_avg"] <= s["k_max"] <= 128
    kinds = {int(h["kind"]) for h, _, _ in iter_ops(P.stream(0, 0), P.page_bytes)}
    assert {1, 6, 8} <= kinds  # gather, interpolation, final blocks written to G
    kinds = {int(h["kind"]) for h, _, _ in iter_ops(P.stream(0, 1), P.page_bytes)}
    assert {2, 3, 7, 9} <= kinds  # scatter, fold, final blocks, anterpolation


def test_rank_property_grows_with_eps():
    """Remark adaptivity: looser eps gives smaller adaptive ranks."""
    a = sht.Plan(128, 1e-12, leaf_cols=16, host_only=True).stats()
    b = sht.Plan(128, 1e-6, leaf_cols=16, host_only=True).stats()
    assert b["k_avg"] < a["k_avg"]
    assert b["factor_values"] < a["factor_values"]


def test_trimming_bounds_dropped_rows():
    """With trimming, dropped rows (a suffix near the poles) have total
    Frobenius norm <= trim_eps, so the transform error stays ~eps."""
    l = 64
    P = sht.Plan(l, 1e-12, leaf_cols=16, trim_eps=1e-8, host_only=True)
    s = P.stats()
    assert s["rows_kept"] < s["rows_total"]
    beta = inputs.random_beta(l, seed=3)
    G = emulate(P.stream(0, 0), P.page_bytes, l, 0, 0, beta)
    assert rel(G, oracle.legendre_synthesis(beta, l)) < 1e-7


@pytest.mark.parametrize("args", [(0, 1e-12), (1025, 1e-12), (8, 0.0), (8, 1.0), (8, -1e-3), (8, float("nan"))])
def test_invalid_arguments_are_rejected(args):
    with pytest.raises(sht.ShtError) as e:
        sht.Plan(*args, host_only=True)
    assert e.value.code == 1


def test_invalid_options_are_rejected():
    for kw in [dict(leaf_cols=1), dict(page_bytes=1000), dict(page_bytes=65536), dict(num_threads=-1),
               dict(consumer_warps=10), dict(slot_values=100), dict(slot_values=4096), dict(slot_values=1000),
               dict(device_build=True), dict(device_build_arena_mb=-1), dict(staging_slots=2),
               dict(values_inline=1), dict(page_bytes=256), dict(page_bytes=8192)]:
        with pytest.raises(sht.ShtError):
            sht.Plan(8, 1e-12, host_only=True, **kw)


def test_host_only_plan_refuses_compute():
    P = sht.Plan(8, 1e-12, host_only=True)
    with pytest.raises(sht.ShtError) as e:
        sht.sht_legendre_synthesize(P, 0, 16, 16, stream=0)
    assert e.value.code == 6


def test_stats_follow_paper_columns():
    """Plan statistics mirror the paper's table columns (Section 5: k_max,
    k_avg, k_sigma, t_quad, t_comp, m_max)."""
    s = sht.Plan(64, 1e-12, leaf_cols=16, host_only=True).stats()
    assert s["l"] == 64 and s["n_units"] == 128
    assert s["t_quad"] >= 0 and s["t_comp"] > 0
    assert s["m_max_words"] > 0
    assert s["factor_flops"] > 0 and s["t_factor"] > 0 and s["t_factor_kernel"] == 0.0
    assert s["k_sigma"] >= 0
    # the strong rank-revealing step of Remark QR_algorithm bounds the
    # interpolation coefficients by 2
    assert s["max_abs_T"] <= 2.0 + 1e-12
    assert math.isfinite(s["k_avg"])


@pytest.mark.parametrize("l,C", [(4, 2), (16, 4), (64, 16), (64, 64)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_op_ordering_is_race_free(l, C, prec):
    """Race detection for the concurrent sweep: every op may overlap the ops
    its `dep` field names; none of them may write what it reads or writes,
    nor read what it writes (sht_stream.h ordering rule).  The split format
    has streams of its own (its ops are cut into other pieces)."""
    P = sht.Plan(l, 1e-12, leaf_cols=C, host_only=True)
    P.prepare(prec)
    for d in (0, 1):
        assert check_races(P.stream(prec, d), P.page_bytes, l) == []


def test_race_checker_catches_a_planted_overlap():
    """The checker itself: dropping the pred entries of the first
    interpolation op that waits for another warp (it would no longer wait for
    the gather that writes its input) must be reported."""
    from tests.stream_emulator import OPHDR
    P = sht.Plan(64, 1e-12, leaf_cols=16, host_only=True)
    records, values = P.stream(0, 0)
    CH = P.page_bytes
    st = (records.copy(), values)
    assert check_races(st, CH, 64) == []
    # locate the record in the copy, walking the items as the decoder does
    pos = 0
    while pos < len(st[0]):
        nw = int(st[0][pos + 4:pos + 6].view("<u2")[0])
        ranges = st[0][pos + 16:pos + 16 + 8 * nw].view("<u4").reshape(nw, 2)
        end = pos
        for w in range(nw):
            off, nb = int(ranges[w, 0]), int(ranges[w, 1])
            end = max(end, pos + off + nb)
            q = 0
            while q < nb:
                at = pos + off + q
                h = st[0][at:at + 32].view(OPHDR)
                if int(h[0]["bytes"]) == 0:
                    q = (q // CH + 1) * CH
                    continue
                if h[0]["kind"] == 6 and int(h[0]["npred"]) > 0:
                    ia = st[0][at + 32:at + 32 + 16 * int(h[0]["idx16"])].view("<u2")
                    npred = int(h[0]["npred"])
                    ia[:len(ia) - npred] = ia[npred:].copy()
                    h[0]["npred"] = 0  # no longer waits for the other warps
                    assert check_races(st, CH, 64) != []
                    return
                q += int(h[0]["bytes"])
        pos = (end + 15) // 16 * 16
    raise AssertionError("no interpolation op that waits for another warp")


def test_every_item_is_scheduled_for_the_plan_warps():
    """Each work item carries one record stream per consumer warp of the plan
    (consumer_warps, 16 by default), and the schedule spreads the ops of a
    large order over many of them."""
    from tests.stream_emulator import iter_items
    for nw in (8, 16):
        P = sht.Plan(128, 1e-12, leaf_cols=16, host_only=True, consumer_warps=nw)
        items = list(iter_items(P.stream(0, 0)[0], P.page_bytes))
        assert items and all(len(w) == nw for w in items)
        # the largest item (both parities of order 0) spreads over at least half of the warps
        assert sum(len(ops) > 0 for ops in items[0]) >= nw // 2


def test_batch_argument_checks_on_host():
    """Batch creation validates its arguments before any CUDA call: empty or
    missing plan lists, bad precisions, and host-only plans are refused."""
    import ctypes
    P = sht.Plan(8, 1e-12, host_only=True)
    L = sht.lib()
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(P.handle)
    assert L.sht_batch_create(0, arr, 0, ctypes.byref(h)) == 1
    assert L.sht_batch_create(1, None, 0, ctypes.byref(h)) == 1
    assert L.sht_batch_create(1, arr, 9, ctypes.byref(h)) == 1
    assert L.sht_batch_create(1, (ctypes.c_void_p * 1)(None), 0, ctypes.byref(h)) == 1
    assert L.sht_batch_create(1, arr, 0, ctypes.byref(h)) == 6  # host-only plan
    assert h.value is None
    assert L.sht_batch_destroy(None) == 0


def test_debug_unmet_dependency_plants_one_self_wait():
    """The failure-detection option makes exactly one compute op per stream
    wait for its own completion (a pred entry naming its own warp and
    position); a normal plan has none."""
    from tests.stream_emulator import OP_ANA, OP_SYN, POS_BITS, iter_items
    for debug, expected in ((1, 1), (0, 0)):
        P = sht.Plan(32, 1e-12, leaf_cols=8, host_only=True, debug_unmet_dependency=debug)
        for d in (0, 1):
            n = 0
            for warps in iter_items(P.stream(0, d)[0], P.page_bytes):
                for w, ops in enumerate(warps):
                    for p, (h, preds, _) in enumerate(ops):
                        if any(int(e) == (w << POS_BITS) | p for e in preds):
                            assert OP_SYN <= int(h["kind"]) <= OP_ANA
                            n += 1
            assert n == expected, (debug, d, n)


def test_plans_do_not_depend_on_the_thread_count():
    """Nodes, weights and the float64 and float32 streams of both directions
    are the same bytes whether the precomputation runs on one host thread, on
    three, or on all of them: every unit and node is computed on its own and
    the streams are laid out in a fixed order."""
    plans = [sht.Plan(128, 1e-12, leaf_cols=16, host_only=True, num_threads=t) for t in (1, 3, 0)]
    ref = plans[0]
    x0, w0 = ref.nodes()
    for P in plans[1:]:
        x, w = P.nodes()
        assert np.array_equal(x, x0) and np.array_equal(w, w0)
        for prec in (0, 1):
            for d in (0, 1):
                for a, b in zip(P.stream(prec, d), ref.stream(prec, d)):
                    assert np.array_equal(a, b), (prec, d)
    for P in plans:
        P.close()


@pytest.mark.parametrize("l,C", [(200, 32), (256, 32)])
def test_split_pieces_need_no_more_ops_than_power_of_two_pieces(l, C):
    """The split format cuts each block into the op pieces its cost estimate
    prefers, float64 into 32, 16, 8, ... outputs, over the same blocks: the
    split streams hold at most as many compute ops (fewer once blocks exceed
    a staging slot), and the same values."""
    from tests.stream_emulator import iter_ops, OP_SYN, OP_ANA
    P = sht.Plan(l, 1e-12, leaf_cols=C, host_only=True)
    P.prepare(2)
    fewer = False
    for d in (0, 1):
        counts, values = [], []
        for prec in (0, 2):
            ops = [h for h, _, _ in iter_ops(P.stream(prec, d), P.page_bytes) if OP_SYN <= int(h["kind"]) <= OP_ANA]
            counts.append(len(ops))
            values.append(sum(int(h["M"]) * int(h["K"]) for h in ops))
        assert counts[1] <= counts[0]
        assert values[1] == values[0]
        fewer |= counts[1] < counts[0]
    assert fewer
