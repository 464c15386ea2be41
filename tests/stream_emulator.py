"""Host emulation of the butterfly factor streams (test code).

Decodes the stream format documented in paper_0910_5435_gb300/csrc/sht_stream.h
(work items whose ops the planner has scheduled onto the CTA's warps, one
record stream per warp) and applies every op with numpy complex128
arithmetic in one valid serialization of the kernel's concurrent execution:
warps advance in turn, an op only once the ops of other warps it lists have
run.  It separates errors of the host precomputation (nodes, recurrence,
IDs, op emission, scheduling) from errors of the CUDA kernels.

``check_races`` verifies the ordering annotations: within a work item an op
is ordered after the earlier ops of its own warp and, through its pred
entries, after ops of other warps (transitively); it may overlap every other
op of the item, so it must neither write anything such an op reads or
writes, nor read anything it writes.
"""

import numpy as np

OPHDR = np.dtype([
    ("bytes", "<u4"), ("kind", "u1"), ("flags", "u1"), ("in_buf", "u1"), ("out_buf", "u1"),
    ("M", "<u2"), ("K", "<u2"), ("nskel", "<u2"), ("io", "<u2"), ("oo", "<u2"), ("npred", "<u2"),
    ("a0", "<u2"), ("idx16", "<u2"), ("a1", "<u4"), ("vref", "<u4"),
])
assert OPHDR.itemsize == 32

OP_GATHER, OP_SCATTER, OP_FOLD, OP_CLEAR, OP_GZERO, OP_SYN, OP_DENSE, OP_DENSE_G, OP_ANA = range(1, 10)
F_ACCUM, F_SKEL = 2, 4
ITEM_MAGIC = 0x53485449
POS_BITS = 12


def iter_items(records, chunk_bytes):
    """The work items of a record region, in order: for each, a list over
    warps of that warp's ops as (header, pred entries, index array)."""
    pos = 0
    n = len(records)
    while pos < n:
        hdr = records[pos:pos + 16].view("<u4")
        if int(hdr[0]) != ITEM_MAGIC:
            if not records[pos:].any():  # trailing padding
                return
            raise AssertionError(f"no item header at byte {pos}")
        nw = int(records[pos + 4:pos + 6].view("<u2")[0])
        ranges = records[pos + 16:pos + 16 + 8 * nw].view("<u4").reshape(nw, 2)
        head = (16 + 8 * nw + 15) // 16 * 16
        end = pos + head
        warps = []
        for w in range(nw):
            off, nb = int(ranges[w, 0]), int(ranges[w, 1])
            assert off % 16 == 0 and nb % 16 == 0, "misaligned warp range"
            st = records[pos + off:pos + off + nb]
            end = max(end, pos + off + nb)
            ops = []
            p = 0
            while p < nb:
                h = st[p:p + 32].view(OPHDR)[0]
                if int(h["bytes"]) == 0:
                    p = (p // chunk_bytes + 1) * chunk_bytes  # rest of the chunk is padding
                    continue
                b = int(h["bytes"])
                assert b >= 32 and b % 16 == 0, "bad record size"
                assert (p % chunk_bytes) + b <= chunk_bytes, "record crosses a chunk boundary"
                ia = st[p + 32:p + 32 + 16 * int(h["idx16"])].view("<u2")
                npred = int(h["npred"])
                ops.append((h, ia[:npred].astype(int), ia[npred:]))
                p += b
            warps.append(ops)
        yield warps
        pos = (end + 15) // 16 * 16


def _serialize(warps):
    """One valid sequential order of an item's ops: (warp, position) pairs."""
    nw = len(warps)
    done = [0] * nw
    order = []
    total = sum(len(x) for x in warps)
    while len(order) < total:
        progressed = False
        for w in range(nw):
            while done[w] < len(warps[w]):
                preds = warps[w][done[w]][1]
                if all(done[e >> POS_BITS] > (e & ((1 << POS_BITS) - 1)) for e in preds):
                    order.append((w, done[w]))
                    done[w] += 1
                    progressed = True
                else:
                    break
        if not progressed:
            raise RuntimeError("the ops of a work item wait for one another in a cycle")
    return order


def iter_ops(stream, chunk_bytes, with_preds=False):
    """Yields (header, index array, value bytes) for every op, work item by
    work item, each item in one valid serialization.  ``stream`` is the
    (records, values) pair of Plan.stream.  With with_preds the index array
    is preceded by the op's pred entries and the header is followed by the
    op's (warp, position): (header, preds, index array, values, (w, p))."""
    records, values = stream
    for warps in iter_items(records, chunk_bytes):
        for w, p in _serialize(warps):
            h, preds, idx = warps[w][p]
            vals = values[16 * int(h["vref"]):] if OP_SYN <= int(h["kind"]) <= OP_ANA else None
            if with_preds:
                yield h, preds, idx, vals, (w, p)
            else:
                yield h, idx, vals


def decode_values(vals, prec, n):
    if prec == 0:
        return vals.view("<f8")[:n].astype(np.float64)
    if prec == 1:
        return vals.view("<f4")[:n].astype(np.float64)
    hl = vals.view("<f4")[:2 * n].astype(np.float64)
    return hl[0::2] + hl[1::2]


def _tri(l):
    L = 2 * l
    return np.concatenate([[0], np.cumsum(L - np.arange(L))])


def emulate(stream, chunk_bytes, l, prec, direction, inp, prescale=None, twiddle=None, plain=False):
    """Applies a whole stream.  direction 0: inp = beta triangle -> G (2l, 2l);
    direction 1: inp = G -> beta triangle.  plain=True applies a single-block
    stream (sht_gj_plan_create: l = n) to vectors of n entries: coefficient
    j and node value r are elements j and r, with no parity interleave,
    fold or unfold (the stages run in their order in the stream)."""
    L = 2 * l
    size = 64 * L + 4096
    bufs = [np.zeros(size, dtype=np.complex128) for _ in range(4)]
    tri = _tri(l)
    if plain:
        tri = np.zeros(L + 1, dtype=np.int64)
    if plain:
        G = None  # single blocks write their node values to y below
        beta = np.asarray(inp, dtype=np.complex128) if direction == 0 else None
    elif direction == 0:
        G = np.full((L, L), np.nan, dtype=np.complex128)
        beta = np.asarray(inp, dtype=np.complex128)
    else:
        beta = np.full(tri[-1], np.nan, dtype=np.complex128)
        G = np.asarray(inp, dtype=np.complex128)
    if plain:
        # a vector of n: the "row" of order 0 at columns l + r, and the
        # coefficients at 2j (p = 0) of a flat array
        if direction == 0:
            y = np.full(l, np.nan, dtype=np.complex128)
            beta2 = np.zeros(2 * l, dtype=np.complex128)
            beta2[0::2] = beta
            beta = beta2
        else:
            y = np.asarray(inp, dtype=np.complex128)
            beta = np.full(2 * l, np.nan, dtype=np.complex128)
    for h, idx, vals in iter_ops(stream, chunk_bytes):
        kind, M, K = int(h["kind"]), int(h["M"]), int(h["K"])
        io, oo = int(h["io"]), int(h["oo"])
        m, p, cb = int(h["a1"]), int(h["a0"]) & 1, int(h["a0"]) >> 1
        src, dst = bufs[int(h["in_buf"])], bufs[int(h["out_buf"])]
        acc = bool(h["flags"] & F_ACCUM)
        tw = 1.0 if twiddle is None else twiddle[m]
        if plain:
            # single blocks: no order; a1 holds the bits of io / oo above 16
            a1 = int(h["a1"])
            io += (a1 & 0xFFFF) << 16
            oo += (a1 >> 16) << 16
            p, m, tw = 0, 0, 1.0
        if plain and kind == OP_FOLD:
            r = oo + np.arange(M)
            dst[cb + oo:cb + oo + M] = y[r]
        elif plain and kind == OP_GZERO:
            y[oo + np.arange(M)] = 0
        elif plain and kind == OP_DENSE_G:
            V = decode_values(vals, prec, K * M).reshape(K, M)
            r = oo + np.arange(M)
            y[r] = (y[r] if acc else 0) + V.T @ src[io:io + K]
        elif kind == OP_GATHER:
            dst[cb + oo:cb + oo + M] = beta[tri[m] + p + 2 * (oo + np.arange(M))]
        elif kind == OP_SCATTER:
            beta[tri[m] + p + 2 * (io + np.arange(M))] = src[cb + io:cb + io + M]
        elif kind == OP_FOLD:
            r = oo + np.arange(M)
            sgn = 1.0 if p == 0 else -1.0
            s = np.ones(M) if prescale is None else prescale[r]
            dst[cb + oo:cb + oo + M] = s * tw * (G[m, l + r] + sgn * G[m, l - 1 - r])
        elif kind == OP_CLEAR:
            dst[oo:oo + M] = 0
        elif kind == OP_GZERO:
            r = oo + np.arange(M)
            G[m, l + r] = 0
            G[m, l - 1 - r] = 0
        elif kind == OP_SYN:
            V = decode_values(vals, prec, K * M).reshape(K, M)
            red = idx[:K].astype(int)
            skel = idx[K:K + M].astype(int)
            dst[oo:oo + M] = V.T @ src[io + red] + src[io + skel]
        elif kind == OP_DENSE:
            V = decode_values(vals, prec, K * M).reshape(K, M)
            dst[oo:oo + M] = V.T @ src[io:io + K]
        elif kind == OP_DENSE_G:
            V = decode_values(vals, prec, K * M).reshape(K, M)
            v = tw * (V.T @ src[io:io + K])
            r = oo + np.arange(M)
            if acc:
                G[m, l + r] += v
                G[m, l - 1 - r] -= v
            else:
                G[m, l + r] = v
                G[m, l - 1 - r] = v
        elif kind == OP_ANA:
            V = decode_values(vals, prec, K * M).reshape(K, M)
            red = idx[:M].astype(int)
            res = V.T @ src[io:io + K]
            if acc:
                dst[oo + red] += res
            else:
                dst[oo + red] = res
            if h["flags"] & F_SKEL:
                nsk = int(h["nskel"])
                skel = idx[M:M + nsk].astype(int)
                if acc:
                    dst[oo + skel] += src[io:io + nsk]
                else:
                    dst[oo + skel] = src[io:io + nsk]
        else:
            raise ValueError(f"unknown op kind {kind}")
    if plain:
        return y if direction == 0 else beta[0::2]
    return G if direction == 0 else beta


def _access_sets(h, idx, l):
    """(reads, writes) of one op as sets of hashable locations."""
    kind, M, K = int(h["kind"]), int(h["M"]), int(h["K"])
    io, oo, m = int(h["io"]), int(h["oo"]), int(h["a1"])
    p, cb = int(h["a0"]) & 1, int(h["a0"]) >> 1
    ib, ob = int(h["in_buf"]), int(h["out_buf"])
    R, W = set(), set()
    if kind == OP_GATHER:
        W |= {("buf", ob, cb + oo + j) for j in range(M)}
        R |= {("beta", m, p + 2 * (oo + j)) for j in range(M)}
    elif kind == OP_SCATTER:
        R |= {("buf", ib, cb + io + j) for j in range(M)}
        W |= {("beta", m, p + 2 * (io + j)) for j in range(M)}
    elif kind == OP_FOLD:
        W |= {("buf", ob, cb + oo + j) for j in range(M)}
        R |= {("G", m, l + oo + j) for j in range(M)} | {("G", m, l - 1 - oo - j) for j in range(M)}
    elif kind == OP_CLEAR:
        W |= {("buf", ob, oo + j) for j in range(M)}
    elif kind == OP_GZERO:
        W |= {("G", m, l + oo + j) for j in range(M)} | {("G", m, l - 1 - oo - j) for j in range(M)}
    elif kind == OP_SYN:
        R |= {("buf", ib, io + int(s)) for s in idx[:K + M]}
        W |= {("buf", ob, oo + o) for o in range(M)}
    elif kind == OP_DENSE:
        R |= {("buf", ib, io + s) for s in range(K)}
        W |= {("buf", ob, oo + o) for o in range(M)}
    elif kind == OP_DENSE_G:
        R |= {("buf", ib, io + s) for s in range(K)}
        rows = {("G", m, l + oo + o) for o in range(M)} | {("G", m, l - 1 - oo - o) for o in range(M)}
        W |= rows
        if h["flags"] & F_ACCUM:
            R |= rows
    elif kind == OP_ANA:
        R |= {("buf", ib, io + s) for s in range(K)}
        outs = {("buf", ob, oo + int(r)) for r in idx[:M]}
        if h["flags"] & F_SKEL:
            nsk = int(h["nskel"])
            outs |= {("buf", ob, oo + int(s)) for s in idx[M:M + nsk]}
        W |= outs
        if h["flags"] & F_ACCUM:
            R |= outs
    return R, W


def check_races(stream, chunk_bytes, l):
    """Returns ((w, p), (w2, p2)) pairs of ops of one item that may overlap
    but conflict."""
    records, _ = stream
    bad = []
    for warps in iter_items(records, chunk_bytes):
        order = _serialize(warps)
        index = {wp: i for i, wp in enumerate(order)}
        anc = [0] * len(order)  # transitive predecessors as int bitsets over serialized positions
        sets = []
        for i, (w, p) in enumerate(order):
            h, preds, idx = warps[w][p]
            a = 0
            if p > 0:
                j = index[(w, p - 1)]
                a |= anc[j] | (1 << j)
            for e in preds:
                we, pe = e >> POS_BITS, e & ((1 << POS_BITS) - 1)
                j = index[(we, pe)]
                a |= anc[j] | (1 << j)
            anc[i] = a
            sets.append(_access_sets(h, idx, l))
            Rt, Wt = sets[-1]
            for j in range(i):
                if (a >> j) & 1:
                    continue
                Ru, Wu = sets[j]
                if (Wt & (Ru | Wu)) or (Rt & Wu):
                    bad.append(((w, p), order[j]))
    return bad


def op_stats(stream, chunk_bytes):
    """Counts ops per kind, for plan diagnostics."""
    counts = {}
    for h, _, _ in iter_ops(stream, chunk_bytes):
        k = int(h["kind"])
        counts[k] = counts.get(k, 0) + 1
    return counts
