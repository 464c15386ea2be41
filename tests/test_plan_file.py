"""Plan files (sht_plan_save / sht_plan_load and the plan_cache option), on
the host: a saved and reloaded plan encodes the same streams, and truncated,
corrupted or foreign files are refused with SHT_ERR_PLAN_CORRUPT."""

import os

import numpy as np
import pytest

from paper_0910_5435_gb300 import sht

CORRUPT, INVALID = 4, 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def same_streams(a, b, precs=(0,)):
    return all(np.array_equal(x, y) for q in precs for d in (0, 1) for x, y in zip(a.stream(q, d), b.stream(q, d)))


@pytest.fixture(scope="module")
def saved(tmp_path_factory):
    P = sht.Plan(64, 1e-12, leaf_cols=16, host_only=True)
    P.prepare(sht.SHT_FP32)
    path = str(tmp_path_factory.mktemp("plans") / "l64.plan")
    P.save(path)
    return P, path


@pytest.mark.parametrize("l,C", [(1, 4), (2, 4), (16, 4), (128, 64)])
def test_round_trip_gives_the_same_streams(tmp_path, l, C):
    P = sht.Plan(l, 1e-12, leaf_cols=C, host_only=True)
    path = str(tmp_path / "p.plan")
    P.save(path)
    Q = sht.Plan.load(path, host_only=True)
    assert Q.l == l
    assert same_streams(P, Q)
    sp, sq = P.stats(), Q.stats()
    for key in ("n_blocks", "k_max", "k_avg", "factor_values", "rows_kept", "m_max_words", "leaf_cols"):
        assert sp[key] == sq[key], key
    assert sq["t_factor"] == 0.0  # nothing was factored


def test_float32_factorization_is_kept_and_options_come_from_the_file(saved):
    P, path = saved
    Q = sht.Plan.load(path, host_only=True, leaf_cols=40, page_bytes=2048)
    s = Q.stats()
    assert s["leaf_cols"] == 16 and s["page_bytes"] == 2048
    Q.prepare(sht.SHT_FP32)
    assert Q.stats()["t_factor"] == 0.0  # the float32 factorization came from the file
    R = sht.Plan.load(path, host_only=True)
    assert same_streams(P, R, precs=(0, 1))


def corrupt_copy(path, tmp_path, edit):
    data = bytearray(open(path, "rb").read())
    data = edit(data)
    out = str(tmp_path / "bad.plan")
    with open(out, "wb") as f:
        f.write(bytes(data))
    return out


@pytest.mark.parametrize("what", ["payload byte", "table byte", "header field", "magic", "version",
                                  "truncated payload", "truncated header", "trailing bytes"])
def test_damaged_files_are_refused(saved, tmp_path, what):
    _, path = saved
    size = os.path.getsize(path)

    def edit(d):
        if what == "payload byte":
            d[size - 1000] ^= 0x40
        elif what == "table byte":
            d[128 + 30] ^= 0x01
        elif what == "header field":
            d[24] ^= 0x01  # min_band_rows
        elif what == "magic":
            d[0:8] = b"NOTAPLAN"
        elif what == "version":
            d[8] = 99
        elif what == "truncated payload":
            d = d[:size - 4096]
        elif what == "truncated header":
            d = d[:100]
        elif what == "trailing bytes":
            d = d + bytes(16)
        return d

    bad = corrupt_copy(path, tmp_path, edit)
    with pytest.raises(sht.ShtError) as e:
        sht.Plan.load(bad, host_only=True)
    assert e.value.code == CORRUPT, what


def test_missing_file_and_unwritable_path(tmp_path):
    with pytest.raises(sht.ShtError) as e:
        sht.Plan.load(str(tmp_path / "none.plan"), host_only=True)
    assert e.value.code == INVALID
    P = sht.Plan(8, 1e-12, leaf_cols=4, host_only=True)
    with pytest.raises(sht.ShtError) as e:
        P.save(str(tmp_path / "no_such_dir" / "p.plan"))
    assert e.value.code == INVALID


def test_plan_cache_builds_once_and_rebuilds_when_stale(tmp_path):
    cache = str(tmp_path / "cache.plan")
    a = sht.Plan(64, 1e-12, leaf_cols=16, host_only=True, plan_cache=cache)
    assert os.path.exists(cache) and a.stats()["t_factor"] > 0
    b = sht.Plan(64, 1e-12, leaf_cols=16, host_only=True, plan_cache=cache)
    assert b.stats()["t_factor"] == 0.0 and same_streams(a, b)
    # other options: the file is not used, and is replaced
    c = sht.Plan(64, 1e-12, leaf_cols=32, host_only=True, plan_cache=cache)
    assert c.stats()["t_factor"] > 0
    d = sht.Plan.load(cache, host_only=True)
    assert d.stats()["leaf_cols"] == 32
    # a damaged cache is rebuilt (and the reason recorded)
    data = bytearray(open(cache, "rb").read())
    data[-100] ^= 0x10
    open(cache, "wb").write(bytes(data))
    e = sht.Plan(64, 1e-12, leaf_cols=32, host_only=True, plan_cache=cache)
    assert e.stats()["t_factor"] > 0 and same_streams(c, e)
    assert b"rebuilt" in sht.lib().sht_last_error_detail()
    sht.Plan.load(cache, host_only=True)  # rewritten intact


def _file_hash(b):
    """The plan file's integrity hash (64-bit multiply-xorshift over
    little-endian 8-byte words, the tail zero-padded), restated so that a test
    can forge a table whose checksums still match."""
    M = (1 << 64) - 1
    n = len(b)
    h = 0x9E3779B97F4A7C15 ^ n
    i = 0
    while i + 8 <= n:
        h = ((h ^ int.from_bytes(b[i:i + 8], "little")) * 0xFF51AFD7ED558CCD) & M
        h ^= h >> 29
        i += 8
    t = int.from_bytes(bytes(b[i:n]) + bytes(8 - (n - i)), "little") if i < n else 0
    h = ((h ^ t) * 0xC4CEB9FE1A85EC53) & M
    return h ^ (h >> 32)


@pytest.mark.parametrize("forgery", ["oversized record", "wrapping sizes"])
def test_forged_unit_table_with_matching_checksums_is_refused(saved, tmp_path, forgery):
    """Record sizes are bounded by the bytes left in the file before anything
    is allocated or hashed: a table whose sizes exceed the file, or wrap
    around 2^64 back to the true total, is refused even when its checksums
    have been recomputed to match."""
    _, path = saved
    d = bytearray(open(path, "rb").read())
    nfact = int.from_bytes(d[12:16], "little")
    units = int.from_bytes(d[28:32], "little")
    nrec = nfact * units
    table = d[128:128 + 24 * nrec]
    assert _file_hash(table) == int.from_bytes(d[56:64], "little")
    hdr = d[:128]
    hdr[64:72] = bytes(8)
    assert _file_hash(hdr) == int.from_bytes(d[64:72], "little")

    recs = [[int.from_bytes(table[24 * r + 8 * j:24 * r + 8 * j + 8], "little") for j in range(3)]
            for r in range(nrec)]
    M = (1 << 64) - 1
    if forgery == "oversized record":
        recs[0][1] += 1 << 40
        for r in range(1, nrec):
            recs[r][0] += 1 << 40
    else:  # two records of about 2^63 bytes each: the sum wraps to the true total
        recs[0][1] += 1 << 63
        recs[1][0] = (recs[1][0] + (1 << 63)) & M
        recs[1][1] = (recs[1][1] + (1 << 63)) & M
    for r in range(nrec):
        for j in range(3):
            table[24 * r + 8 * j:24 * r + 8 * j + 8] = recs[r][j].to_bytes(8, "little")
    d[128:128 + 24 * nrec] = table
    d[56:64] = _file_hash(table).to_bytes(8, "little")
    hdr = d[:128]
    hdr[64:72] = bytes(8)
    d[64:72] = _file_hash(hdr).to_bytes(8, "little")
    bad = corrupt_copy(path, tmp_path, lambda _: d)
    with pytest.raises(sht.ShtError) as e:
        sht.Plan.load(bad, host_only=True)
    assert e.value.code == CORRUPT
    assert b"payload ends early" in sht.lib().sht_last_error_detail()


def test_forged_block_count_is_refused_before_allocation(saved, tmp_path):
    """A unit record claiming more ID blocks than its remaining bytes can hold
    (each serialized block takes at least 64 bytes) is refused as implausible
    before the blocks are allocated, even with every checksum recomputed."""
    _, path = saved
    d = bytearray(open(path, "rb").read())
    nrec = int.from_bytes(d[12:16], "little") * int.from_bytes(d[28:32], "little")
    t0 = 128
    p0 = t0 + 24 * nrec  # payload start; record 0 is the float64 unit m = 0, p = 0
    off, nbytes = (int.from_bytes(d[t0 + 8 * j:t0 + 8 * j + 8], "little") for j in range(2))
    at = p0 + off + 6 * 4 + 4 * 8 + 8  # after m, p, n, rows, direct, levels, four counts, cost
    nD = int.from_bytes(d[at:at + 8], "little")
    at += 8 + 8 * nD
    nw = int.from_bytes(d[at:at + 8], "little")
    at += 8 + 4 * nw
    nb = int.from_bytes(d[at:at + 8], "little")
    assert 0 < nb < 1000  # the unit is a butterfly with a plausible block count
    left = p0 + off + nbytes - (at + 8)
    d[at:at + 8] = (left // 64 + 1).to_bytes(8, "little")
    d[t0 + 16:t0 + 24] = _file_hash(d[p0 + off:p0 + off + nbytes]).to_bytes(8, "little")
    d[56:64] = _file_hash(d[t0:p0]).to_bytes(8, "little")
    hdr = d[:128]
    hdr[64:72] = bytes(8)
    d[64:72] = _file_hash(hdr).to_bytes(8, "little")
    bad = corrupt_copy(path, tmp_path, lambda _: d)
    with pytest.raises(sht.ShtError) as e:
        sht.Plan.load(bad, host_only=True)
    assert e.value.code == CORRUPT
    assert b"implausible block count" in sht.lib().sht_last_error_detail()


def test_version_1_files_are_refused_and_rebuilt_as_a_cache(tmp_path):
    """Files of format version 1 hold factorizations of the earlier quadrature
    weights: with a valid header checksum they are still refused, and given as
    a plan_cache they are rebuilt and rewritten at the current version."""
    cache = str(tmp_path / "v1.plan")
    a = sht.Plan(16, 1e-12, leaf_cols=4, host_only=True, plan_cache=cache)
    d = bytearray(open(cache, "rb").read())
    assert int.from_bytes(d[8:12], "little") == 2
    d[8:12] = (1).to_bytes(4, "little")
    hdr = d[:128]
    hdr[64:72] = bytes(8)
    d[64:72] = _file_hash(hdr).to_bytes(8, "little")
    open(cache, "wb").write(bytes(d))
    with pytest.raises(sht.ShtError) as e:
        sht.Plan.load(cache, host_only=True)
    assert e.value.code == CORRUPT and b"version" in sht.lib().sht_last_error_detail()
    b = sht.Plan(16, 1e-12, leaf_cols=4, host_only=True, plan_cache=cache)
    assert b.stats()["t_factor"] > 0 and same_streams(a, b)
    assert int.from_bytes(open(cache, "rb").read()[8:12], "little") == 2
