"""Host emulation of the butterfly factor streams (test code).

Decodes the page format documented in paper_0910_5435_gb300/csrc/sht_stream.h
and applies every op with numpy complex128 arithmetic, in stream order.  It
separates errors of the host precomputation (nodes, recurrence, IDs, op
emission) from errors of the CUDA kernels: the kernels must reproduce this
emulation up to float rounding.
"""

import numpy as np

OPHDR = np.dtype([
    ("bytes", "<u4"), ("kind", "u1"), ("flags", "u1"), ("in_buf", "u1"), ("out_buf", "u1"),
    ("M", "<u2"), ("K", "<u2"), ("nskel", "<u2"), ("io", "<u2"), ("oo", "<u2"), ("a0", "<u2"),
    ("a1", "<u4"), ("idx_bytes", "<u4"), ("pad", "<u4"),
])
assert OPHDR.itemsize == 32

OP_GATHER, OP_SCATTER, OP_UNFOLD, OP_FOLD, OP_CLEAR, OP_SYN, OP_DENSE, OP_ANA = range(1, 9)
OP_QUIT = 0xFF
F_SYNC, F_ACCUM, F_SKEL = 1, 2, 4
BUF_A, BUF_B, BUF_E, BUF_O = range(4)


def iter_ops(stream, page_bytes):
    """Yields (header, index array, value bytes) for every op, in order."""
    npages = len(stream) // page_bytes
    for pg in range(npages):
        page = stream[pg * page_bytes:(pg + 1) * page_bytes]
        off = 0
        while off + 32 <= page_bytes:
            h = page[off:off + 32].view(OPHDR)[0]
            if h["bytes"] == 0:
                break
            if h["kind"] == OP_QUIT:
                return
            ib = int(h["idx_bytes"])
            idx = page[off + 32:off + 32 + ib].view("<u2")
            vals = page[off + 32 + ib:off + int(h["bytes"])]
            yield h, idx, vals
            off += int(h["bytes"])


def decode_values(vals, prec, n):
    if prec == 0:
        return vals.view("<f8")[:n].astype(np.float64)
    if prec == 1:
        return vals.view("<f4")[:n].astype(np.float64)
    hl = vals.view("<f4")[:2 * n].astype(np.float64)
    return hl[0::2] + hl[1::2]


def emulate(stream, page_bytes, l, prec, direction, inp, prescale=None):
    """Applies a whole stream.  direction 0: inp = beta triangle -> G (2l, 2l);
    direction 1: inp = G -> beta triangle."""
    L = 2 * l
    size = 8 * L + 64
    bufs = [np.zeros(size, dtype=np.complex128) for _ in range(4)]
    tri = np.concatenate([[0], np.cumsum(L - np.arange(L))])
    if direction == 0:
        out = np.zeros((L, L), dtype=np.complex128)
        beta = np.asarray(inp, dtype=np.complex128)
    else:
        out = np.zeros(tri[-1], dtype=np.complex128)
        G = np.asarray(inp, dtype=np.complex128)
    for h, idx, vals in iter_ops(stream, page_bytes):
        kind, M, K = int(h["kind"]), int(h["M"]), int(h["K"])
        io, oo = int(h["io"]), int(h["oo"])
        m = int(h["a1"])
        src, dst = bufs[int(h["in_buf"])], bufs[int(h["out_buf"])]
        if kind == OP_GATHER:
            p = int(h["a0"])
            dst[oo:oo + M] = beta[tri[m] + p + 2 * np.arange(M)]
        elif kind == OP_SCATTER:
            p = int(h["a0"])
            out[tri[m] + p + 2 * np.arange(M)] = src[io:io + M]
        elif kind == OP_UNFOLD:
            E = np.zeros(l, dtype=np.complex128)
            O = np.zeros(l, dtype=np.complex128)
            E[:M] = bufs[BUF_E][:M]
            O[:K] = bufs[BUF_O][:K]
            out[m, l:] = E + O
            out[m, :l] = (E - O)[::-1]
        elif kind == OP_FOLD:
            gp = G[m, l:]
            gm = G[m, :l][::-1]
            s = np.ones(l) if prescale is None else prescale
            bufs[BUF_E][:l] = s * (gp + gm)
            bufs[BUF_O][:l] = s * (gp - gm)
        elif kind == OP_CLEAR:
            dst[oo:oo + M] = 0
        elif kind == OP_SYN:
            V = decode_values(vals, prec, K * M).reshape(K, M)
            red = idx[:K].astype(int)
            nsk = int(h["nskel"])
            skel = idx[K:K + nsk].astype(int)
            acc = V.T @ src[io + red]
            if nsk:
                acc[:nsk] += src[io + skel]
            if h["flags"] & F_ACCUM:
                dst[oo:oo + M] += acc
            else:
                dst[oo:oo + M] = acc
        elif kind == OP_DENSE:
            V = decode_values(vals, prec, K * M).reshape(K, M)
            acc = V.T @ src[io:io + K]
            if h["flags"] & F_ACCUM:
                dst[oo:oo + M] += acc
            else:
                dst[oo:oo + M] = acc
        elif kind == OP_ANA:
            V = decode_values(vals, prec, K * M).reshape(K, M)
            red = idx[:M].astype(int)
            acc = V.T @ src[io:io + K]
            np.add.at(dst, oo + red, acc)
            if h["flags"] & F_SKEL:
                nsk = int(h["nskel"])
                skel = idx[M:M + nsk].astype(int)
                np.add.at(dst, oo + skel, src[io:io + nsk])
        else:
            raise ValueError(f"unknown op kind {kind}")
    return out


def op_stats(stream, page_bytes):
    """Counts ops per kind and value bytes, for plan diagnostics."""
    counts = {}
    for h, _, vals in iter_ops(stream, page_bytes):
        k = int(h["kind"])
        counts[k] = counts.get(k, 0) + 1
    return counts
