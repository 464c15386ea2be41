"""Single-block butterflies (sht_unit_stats_compute, host only): their
errors against the direct products, and, for the m = 0 even block, the
rank statistics beside those the paper prints (Section 5, Table small_time
and Table small_pre; tests/golden/paper_small_tables.txt).

At m = 0, parity 0 and n = l the block sqrt(2 w_{l+i}) P-bar^0_{2j}(x_{l+i})
is the paper's even-degree matrix (its weights rho_i are 2 w_{l+i}).  The
rank rule, leaf partition and band splitting here are this library's own,
so the paper's numbers are matched in magnitude and trend, not exactly:
the tolerances below say how closely.
"""

import os

import pytest

from paper_0910_5435_gb300 import sht

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_small_tables.txt")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def paper_rows():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        n, m, kmax, kavg, ksig, efwd, einv = line.split()
        rows[int(n)] = dict(k_max=int(kmax), k_avg=float(kavg), k_sigma=float(ksig),
                            eps_fwd=float(efwd), eps_inv=float(einv))
    return rows


@pytest.mark.parametrize("l,m,p", [(64, 0, 0), (64, 5, 1), (100, 37, 0), (200, 150, 1)])
def test_block_errors_within_id_precision(l, m, p):
    """The butterfly and its transpose agree with the direct products to a
    small multiple of eps_id on unit-norm inputs (Section 2.1 eq. 2.1 bound,
    summed over the levels)."""
    eps = 1e-12
    s = sht.unit_stats(l, m, p, eps_id=eps, leaf_cols=16)
    assert s["n"] == (2 * l - m - p + 1) // 2
    assert s["eps_fwd"] < 50 * eps and s["eps_inv"] < 50 * eps
    # an ID's rank is at most the block's smaller dimension
    assert 0 < s["k_max"] <= min(s["n"], s["rows_kept"]) or s["direct"] == 1


def test_tighter_threshold_raises_ranks_and_lowers_errors():
    a = sht.unit_stats(400, 0, 0, eps_id=1e-10, leaf_cols=32)
    b = sht.unit_stats(400, 0, 0, eps_id=1e-14, leaf_cols=32)
    assert b["k_avg"] > a["k_avg"] and b["factor_values"] > a["factor_values"]
    assert b["eps_fwd"] < a["eps_fwd"] and b["eps_inv"] < a["eps_inv"]


def test_m0_even_block_beside_paper_table_n1250():
    """n = l = 1250, m = 0, even degrees, leaf width C = 60 as in Section 5,
    IDs to nearly machine precision (eps_id = 1e-15).  Printed: k_max 110,
    k_avg 67.0, k_sigma 23.3, eps_fwd 0.49e-14, eps_inv 0.12e-12, m_max
    0.86e6.  Here: the average rank within 20 %, the maximum within 25 %,
    m_max within a factor 2, and both errors at or below the printed ones."""
    ref = paper_rows()[1250]
    s = sht.unit_stats(1250, 0, 0, eps_id=1e-15, leaf_cols=60)
    assert s["n"] == 1250
    assert abs(s["k_avg"] - ref["k_avg"]) <= 0.20 * ref["k_avg"], s["k_avg"]
    assert abs(s["k_max"] - ref["k_max"]) <= 0.25 * ref["k_max"], s["k_max"]
    assert 0.43e6 <= s["m_max_words"] <= 1.72e6, s["m_max_words"]
    assert s["eps_fwd"] <= ref["eps_fwd"] and s["eps_inv"] <= ref["eps_inv"]


def test_invalid_arguments():
    import ctypes
    out = sht.sht_unit_stats()
    L = sht.lib()
    for args in [(0, 0, 0, 1e-12), (40001, 0, 0, 1e-12), (64, 128, 0, 1e-12), (64, 0, 2, 1e-12), (64, 0, 0, 0.0)]:
        assert L.sht_unit_stats_compute(*args, None, 1, ctypes.byref(out)) == 1
