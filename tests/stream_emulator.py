"""Host emulation of the butterfly factor streams (test code).

Decodes the page format documented in paper_0910_5435_gb300/csrc/sht_stream.h
and applies every op with numpy complex128 arithmetic, in stream order (a
valid serialization of the kernel's concurrent execution).  It separates
errors of the host precomputation (nodes, recurrence, IDs, op emission) from
errors of the CUDA kernels.

``check_races`` verifies the ordering annotations: within a work item (opened
by a JOIN that waits for everything before it), op t may overlap every earlier
op that is not among its transitive predecessors, so it must neither write
anything such an op reads or writes, nor read anything it writes.
"""

import numpy as np

OPHDR = np.dtype([
    ("bytes", "<u4"), ("kind", "u1"), ("flags", "u1"), ("in_buf", "u1"), ("out_buf", "u1"),
    ("M", "<u2"), ("K", "<u2"), ("nskel", "<u2"), ("io", "<u2"), ("oo", "<u2"), ("npred", "<u2"),
    ("a0", "<u2"), ("idx16", "<u2"), ("a1", "<u4"), ("vref", "<u4"),
])
assert OPHDR.itemsize == 32

OP_GATHER, OP_SCATTER, OP_FOLD, OP_CLEAR, OP_GZERO, OP_SYN, OP_DENSE, OP_DENSE_G, OP_ANA, OP_JOIN = range(1, 11)
OP_QUIT = 0xFF
F_ACCUM, F_SKEL, F_ITEM_START, F_VALUES_APART = 2, 4, 8, 16


QUIT_PAGE = 0xFFFF


def page_op_offsets(page, page_bytes):
    """Byte offsets of a page's ops from its op table (None for the final
    page): the uint16 at page_bytes - 2 is the count, the uint16 at
    page_bytes - 4 - 2 i the offset of op i in 16-byte units."""
    n = int(page[page_bytes - 2:page_bytes].view("<u2")[0])
    if n == QUIT_PAGE:
        return None
    tab = page[page_bytes - 2 - 2 * n:page_bytes - 2].view("<u2")[::-1]
    return [16 * int(o) for o in tab]


def iter_ops(stream, page_bytes, with_preds=False):
    """Yields (header, index array, value bytes) for every op, in order.
    ``stream`` is the (pages, values) pair of Plan.stream (or the page region
    alone); the index array excludes the leading predecessor deltas unless
    with_preds."""
    if isinstance(stream, tuple):
        pages, values = stream
    else:
        pages, values = stream, None
    npages = len(pages) // page_bytes
    for pg in range(npages):
        page = pages[pg * page_bytes:(pg + 1) * page_bytes]
        offs = page_op_offsets(page, page_bytes)
        if offs is None:
            return
        end = 0
        for off in offs:
            assert off == end, "op table does not chain the ops contiguously"
            h = page[off:off + 32].view(OPHDR)[0]
            assert h["bytes"] > 0 and h["kind"] != OP_QUIT
            end = off + int(h["bytes"])
            assert end <= page_bytes - 2 - 2 * len(offs), "op runs into the op table"
            ib = 16 * int(h["idx16"])
            idx = page[off + 32:off + 32 + ib].view("<u2")
            if not with_preds:
                idx = idx[int(h["npred"]):]
            if h["flags"] & F_VALUES_APART:
                vals = values[16 * int(h["vref"]):]
            else:
                vals = page[off + 32 + ib:off + int(h["bytes"])]
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


def emulate(stream, page_bytes, l, prec, direction, inp, prescale=None, twiddle=None):
    """Applies a whole stream.  direction 0: inp = beta triangle -> G (2l, 2l);
    direction 1: inp = G -> beta triangle."""
    L = 2 * l
    size = 8 * L + 64
    bufs = [np.zeros(size, dtype=np.complex128) for _ in range(4)]
    tri = _tri(l)
    if direction == 0:
        G = np.full((L, L), np.nan, dtype=np.complex128)
        beta = np.asarray(inp, dtype=np.complex128)
    else:
        beta = np.full(tri[-1], np.nan, dtype=np.complex128)
        G = np.asarray(inp, dtype=np.complex128)
    for h, idx, vals in iter_ops(stream, page_bytes):
        kind, M, K = int(h["kind"]), int(h["M"]), int(h["K"])
        io, oo = int(h["io"]), int(h["oo"])
        m, p, cb = int(h["a1"]), int(h["a0"]) & 1, int(h["a0"]) >> 1
        src, dst = bufs[int(h["in_buf"])], bufs[int(h["out_buf"])]
        acc = bool(h["flags"] & F_ACCUM)
        tw = 1.0 if twiddle is None else twiddle[m]
        if kind == OP_JOIN:
            continue
        if kind == OP_GATHER:
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


def check_races(stream, page_bytes, l):
    """Returns (t, u) op pairs (stream positions) that may overlap but conflict."""
    ops = list(iter_ops(stream, page_bytes, with_preds=True))
    bad = []
    start = 0
    while start < len(ops):
        end = start + 1
        while end < len(ops) and not (ops[end][0]["kind"] == OP_JOIN and ops[end][0]["flags"] & F_ITEM_START):
            end += 1
        anc = []  # transitive predecessors (positions within the item) as int bitsets
        sets = []
        for t in range(start, end):
            h, idx, _ = ops[t]
            npred = int(h["npred"])
            a = 0
            for d in idx[:npred]:
                u = t - int(d) - start
                assert 0 <= u < t - start, "predecessor outside its work item"
                a |= anc[u] | (1 << u)
            anc.append(a)
            sets.append(_access_sets(h, idx[npred:], l))
            Rt, Wt = sets[-1]
            for u in range(t - start):
                if (a >> u) & 1:
                    continue
                Ru, Wu = sets[u]
                if (Wt & (Ru | Wu)) or (Rt & Wu):
                    bad.append((t, start + u))
        start = end
    return bad


def op_stats(stream, page_bytes):
    """Counts ops per kind, for plan diagnostics."""
    counts = {}
    for h, _, _ in iter_ops(stream, page_bytes):
        k = int(h["kind"])
        counts[k] = counts.get(k, 0) + 1
    return counts
