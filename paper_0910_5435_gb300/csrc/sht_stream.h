// sht_stream.h -- device layout of the butterfly factor streams.
//
// Shared by the host-side emitter (plan_build.cpp) and the sweep kernels
// (sweep.cu).  One stream exists per (precision, direction); direction 0 is
// synthesis (coefficients -> node values), 1 is analysis (the transposed
// application, Section 2.2 remark after Figure multi).
//
// A stream is a sequence of fixed-size PAGES (page_bytes each, the unit of
// one TMA bulk copy), plus, for plans that keep values apart, a VALUE REGION
// that the executing warp reads directly (coalesced streaming loads): then
// pages carry only headers and index lists, so the ring of pages in shared
// memory spans many more ops.  A work item (one large order m, or several small
// ones) owns a contiguous run of pages; the item table lists them in
// decreasing size (LPT order for the persistent kernel's work queue).  A
// page holds a sequence of OPS, each 16-byte aligned:
//
//   [OpHdr 32 B][uint16 index lists, padded to 16 B][values, padded to 16 B]
//
// from offset 0 up, and ends with an OP TABLE that grows down from the page
// end: the uint16 at byte page_bytes - 2 is the op count n (kQuitPage marks
// the final page), and the uint16 at byte page_bytes - 4 - 2 i is the offset
// of op i in 16-byte units.  The table lets a whole warp publish a page's
// ops at once.  Between the last op and the table the page is zero.
//
// Every op is executed by ONE warp.  Compute ops apply a small dense matrix V
// ([K][M] layout, M fastest: lanes that own consecutive outputs read
// consecutive values) to a vector held in shared memory; M <= 32:
//
//   SYN_INTERP  out[oo + o] = in[io + skel[o]] + sum_s V[s][o] in[io + red[s]]
//               -- one interpolation matrix of an ID (Section 2.1 eq. 2.1,
//               Section 2.2 eqs. 1-6: y = z[skel] + T z[red]);
//   DENSE       out[oo + o] = sum_s V[s][o] in[io + s]
//               -- stored skeleton columns (the unprocessed blocks of
//               Section 3) or a dense block, into shared memory;
//   DENSE_G     the same, written to the node values of order m: with
//               v_i = sum_s V[s][o] in[io + s], i = oo + o, the parity unfold
//               of Section 2.3: G[m][l+i] (= or +=) v_i, G[m][l-1-i] (= or -=) v_i
//               (F_ACCUM for the odd parity, after the even one has written);
//   ANA_INTERP  out[oo + red[o]] (= or +=) sum_s V[s][o] in[io + s], and with
//               F_SKEL also out[oo + skel[t]] (= or +=) in[io + t]
//               -- the transpose of an interpolation matrix (anterpolation).
//
// Control ops carry no values and cover an element range [start, start + M):
// GATHER / SCATTER move one parity of beta^m between global and shared
// memory, FOLD forms u_i = s_i (G[m][l+i] +- G[m][l-1-i]) (the parity fold),
// CLEAR zeroes a shared range, GZERO zeroes node rows of G.
//
// Placement: each parity block's ops address the shared vectors from a base
// position the planner chose for the block, so that consecutive blocks of a
// work item use disjoint ranges where they fit and run concurrently.  Compute
// ops and CLEAR carry the base in io / oo; GATHER, SCATTER and FOLD, whose
// offsets also index coefficients or node rows, carry it in a0 >> 1 (a0 & 1
// is the parity) and address vector position base + j for element j.
//
// Ordering: ops are numbered in stream order (per CTA).  Op t lists its
// predecessors as npred deltas d (op t - d) at the start of its index area:
// the last writer of every shared position / node row it reads or writes and
// every reader of a position it overwrites.  It starts once they have all
// completed, so independent blocks (one butterfly level, the two halves of a
// merge, consecutive orders of one work item) run concurrently.  A work item
// opens with a JOIN (F_ITEM_START) that waits for every earlier op; ops with
// no other predecessor depend on it.  Deltas stay below kDoneWindow.
//
// Values: float64 (SHT_FP64), float2 {hi, lo} (SHT_SPLIT32) or float
// (SHT_FP32).  Shared-memory vectors hold complex numbers in the working
// format of the precision (double2, float4 {re_hi, re_lo, im_hi, im_lo} or
// float2), indexed in elements.

#pragma once
#include <stdint.h>

namespace sht {

enum OpKind : uint8_t {
  OP_END = 0,
  OP_GATHER = 1,      // buf[out_buf][b + j] = beta^m_{m+p+2j}, j in [oo, oo + M)  (a0 = p | b << 1, a1 = m)
  OP_SCATTER = 2,     // beta^m_{m+p+2j} = buf[in_buf][b + j], j in [io, io + M)   (a0 = p | b << 1, a1 = m)
  OP_FOLD = 3,        // buf[out_buf][b + r] = s (G[m][l+r] + (-1)^p G[m][l-1-r]), r in [oo, oo + M)
  OP_CLEAR = 4,       // buf[out_buf][oo + j] = 0, j < M
  OP_GZERO = 5,       // G[m][l+r] = G[m][l-1-r] = 0, r = oo + j, j < M            (a1 = m)
  OP_SYN_INTERP = 6,
  OP_DENSE = 7,
  OP_DENSE_G = 8,     // (a1 = m)
  OP_ANA_INTERP = 9,
  OP_JOIN = 10,       // no data; completes when its predecessors have (F_ITEM_START: when
                      //   every earlier op of the CTA has)
  OP_QUIT = 0xFF,
};

enum OpFlags : uint8_t {
  F_ACCUM = 2,        // DENSE_G / ANA_INTERP: accumulate instead of overwrite
  F_SKEL = 4,         // ANA_INTERP: also the skeleton pass-through (nskel entries)
  F_ITEM_START = 8,   // JOIN opening a work item
  F_VALUES_APART = 16,  // the value block lives in the stream's value region (see vref)
};

struct alignas(16) OpHdr {
  uint32_t bytes;     // size of this op in the page (multiple of 16); 0 terminates the page
  uint8_t kind;
  uint8_t flags;
  uint8_t in_buf;     // shared-memory vector ids 0..3
  uint8_t out_buf;
  uint16_t M;         // outputs (compute ops, <= 32) or element count (control ops)
  uint16_t K;         // inner dimension
  uint16_t nskel;     // SYN_INTERP: M; ANA_INTERP with F_SKEL: pass-through inputs
  uint16_t io;        // element offset of the input vector
  uint16_t oo;        // element offset of the output vector / start of a control range
  uint16_t npred;     // predecessor count; the deltas lead the index area (see above)
  uint16_t a0;        // GATHER / SCATTER / FOLD: parity | vector base << 1
  uint16_t idx16;     // bytes of the index area / 16
  uint32_t a1;        // order m
  uint32_t vref;      // F_VALUES_APART: offset of the value block in the value region, in
                      //   16-byte units; otherwise the values follow the index area
};
static_assert(sizeof(OpHdr) == 32, "OpHdr must be 32 bytes");

// Index area contents (uint16): pred[npred] (deltas), then, with offsets
// relative to io / oo:
//   SYN_INTERP: red[K] then skel[M]
//   ANA_INTERP: red[M] then (F_SKEL) skel[nskel]
//   others:     none

struct UnitEntry {
  uint64_t first_page;  // index of the item's first page in the stream
  uint32_t n_pages;
  uint32_t m;           // first order of the item (informational)
};
static_assert(sizeof(UnitEntry) == 16, "UnitEntry must be 16 bytes");

// Shared-memory vectors A (id 0) and B (id 1), each buf_ab complex elements;
// the butterfly levels alternate between them, and the two parities of an
// order use them one after the other.
constexpr int kNumVecs = 2;

constexpr int kMaxM = 32;             // outputs per compute op (one warp)
constexpr int kMaxPred = 32;          // predecessors listed by a data op (more: fan-in JOIN); one warp checks 32 at once
constexpr int kDoneWindow = 4096;     // completion-tag ring; a segment (ops after an item-start JOIN) holds < kMaxItemOps ops
constexpr int kMaxItemOps = 3584;
// F_VALUES_APART: default cap on the values of one op, which fill one warp's
// staging slot (a plan option).  Smaller slots let more warps fit in shared
// memory but split the blocks into more ops.
constexpr int kDefaultSlotValues = 1024;
constexpr int kMinSlotValues = 128;
constexpr int kMaxSlotValues = 2048;
constexpr int kCtlPieces = 8;         // control ops are split into up to this many warp tasks
constexpr uint16_t kQuitPage = 0xFFFF;  // op count of the stream's final page

// Op table of a page (see the format above).
inline size_t page_table_bytes(int n_ops) { return 2 * (size_t)(n_ops + 1); }

}  // namespace sht
