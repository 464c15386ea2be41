// sht_stream.h -- device layout of the butterfly factor streams.
//
// Shared by the host-side emitter (plan_build.cpp) and the sweep kernels
// (sweep.cu).  One stream exists per (precision, direction); direction 0 is
// synthesis (coefficients -> node values), 1 is analysis (the transposed
// application, Section 2.2 remark after Figure multi).
//
// A stream has a RECORD REGION and a VALUE REGION.  The record region is a
// sequence of WORK ITEMS (one large order m, or several small ones), each
// starting on a 16-byte boundary; the item table lists them in decreasing
// size (LPT order for the persistent kernel's work queue).  The planner has
// already SCHEDULED every op of an item onto one of the nw consumer warps of
// a CTA (list scheduling over the item's dependency graph, plan option
// consumer_warps), so an item holds one record stream per warp:
//
//   ItemHeader (16 B) | WarpRange[nw] (8 B each), padded to 16 B |
//   warp 0's records | warp 1's records | ...
//
// A warp's records are fetched in CHUNKS of chunk_bytes (the plan option
// page_bytes) by 1-D bulk copies into a two-chunk ring of its own; no record
// crosses a chunk boundary, and a record header with bytes == 0 ends a
// chunk early (the rest of it is padding).  A record is
//
//   [OpHdr 32 B][uint16 preds[npred]][uint16 index lists], padded to 16 B
//
// and its values, if any, are a block of the value region (vref) that the
// warp bulk-copies into its staging slot before the op runs.
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
// Ordering: a warp runs its records in order.  A record lists the ops of
// OTHER warps it must wait for, one entry per warp at most: pred = (w << 12)
// | p means "warp w has completed its ops 0..p of this item" (the last
// writer of every shared position / node row the op reads or writes and
// every reader of a position it overwrites, reduced to the latest such op of
// each warp).  After an op flagged F_PUBLISH (one that another warp waits
// for) a warp publishes its progress in shared memory; an item ends with a
// CTA-wide barrier (the next item reuses the shared vectors).
// Each warp's list is in one topological order of the item's graph, so the
// waits cannot form a cycle.
//
// Values: float64 (SHT_FP64), float2 {hi, lo} (SHT_SPLIT32) or float
// (SHT_FP32).  Shared-memory vectors hold complex numbers in the working
// format of the precision (double2, float4 {re_hi, re_lo, im_hi, im_lo} or
// float2), indexed in elements.

#pragma once
#include <stdint.h>

namespace sht {

enum OpKind : uint8_t {
  OP_END = 0,         // bytes == 0: the rest of the chunk is padding
  OP_GATHER = 1,      // buf[out_buf][b + j] = beta^m_{m+p+2j}, j in [oo, oo + M)  (a0 = p | b << 1, a1 = m)
  OP_SCATTER = 2,     // beta^m_{m+p+2j} = buf[in_buf][b + j], j in [io, io + M)   (a0 = p | b << 1, a1 = m)
  OP_FOLD = 3,        // buf[out_buf][b + r] = s (G[m][l+r] + (-1)^p G[m][l-1-r]), r in [oo, oo + M)
  OP_CLEAR = 4,       // buf[out_buf][oo + j] = 0, j < M
  OP_GZERO = 5,       // G[m][l+r] = G[m][l-1-r] = 0, r = oo + j, j < M            (a1 = m)
  OP_SYN_INTERP = 6,
  OP_DENSE = 7,
  OP_DENSE_G = 8,     // (a1 = m)
  OP_ANA_INTERP = 9,
};

enum OpFlags : uint8_t {
  F_ACCUM = 2,        // DENSE_G / ANA_INTERP: accumulate instead of overwrite
  F_SKEL = 4,         // ANA_INTERP: also the skeleton pass-through (nskel entries)
  F_PUBLISH = 8,      // another warp waits for this op: publish the warp's progress after it
};

struct alignas(16) OpHdr {
  uint32_t bytes;     // size of this record (multiple of 16); 0 ends the chunk
  uint8_t kind;
  uint8_t flags;
  uint8_t in_buf;     // shared-memory vector ids 0..3
  uint8_t out_buf;
  uint16_t M;         // outputs (compute ops, <= 32) or element count (control ops)
  uint16_t K;         // inner dimension
  uint16_t nskel;     // SYN_INTERP: M; ANA_INTERP with F_SKEL: pass-through inputs
  uint16_t io;        // element offset of the input vector
  uint16_t oo;        // element offset of the output vector / start of a control range
  uint16_t npred;     // entries of preds[]
  uint16_t a0;        // GATHER / SCATTER / FOLD: parity | vector base << 1
  uint16_t idx16;     // bytes of the index area (preds and index lists) / 16
  uint32_t a1;        // order m; single-block (plain) streams: the bits of io (low half) and oo (high half) above 16
  uint32_t vref;      // compute ops: offset of the value block in the value region, in 16-byte units
};
static_assert(sizeof(OpHdr) == 32, "OpHdr must be 32 bytes");

// Index area contents (uint16): preds[npred], then, with offsets relative
// to io / oo:
//   SYN_INTERP: red[K] then skel[M]
//   ANA_INTERP: red[M] then (F_SKEL) skel[nskel]
//   others:     none

constexpr uint32_t kItemMagic = 0x53485449u;  // "ITHS"
struct ItemHeader {
  uint32_t magic;
  uint16_t nw;        // consumer warps the item was scheduled for
  uint16_t reserved;
  uint32_t n_ops;
  uint32_t reserved2;
};
static_assert(sizeof(ItemHeader) == 16, "ItemHeader must be 16 bytes");
struct WarpRange {
  uint32_t off;       // bytes from the item start (multiple of 16)
  uint32_t bytes;     // length of the warp's record stream (multiple of 16; 0: no ops)
};

struct UnitEntry {
  uint64_t off16;     // byte offset of the item in the record region / 16
  uint32_t len16;     // item bytes / 16
  uint32_t m;         // first order of the item (informational); batches: the field
};
static_assert(sizeof(UnitEntry) == 16, "UnitEntry must be 16 bytes");

// Shared-memory vectors A (id 0) and B (id 1), each buf_ab complex elements;
// the butterfly levels alternate between them.
constexpr int kNumVecs = 2;

constexpr int kMaxM = 32;             // outputs per compute op (one warp)
constexpr int kMaxWarps = 16;         // consumer warps a plan can be scheduled for
constexpr int kPredPosBits = 12;      // pred entry: (warp << 12) | position
constexpr int kMaxWarpOps = (1 << kPredPosBits) - 1;  // ops of one warp in one item
// Default cap on the values of one op: one warp's 8 KB staging slot of 8-byte
// values (the planner doubles it for 4-byte float32 values).  Smaller slots
// let more warps fit in shared memory but split the blocks into more ops.
constexpr int kDefaultSlotValues = 1024;
constexpr int kMinSlotValues = 128;
constexpr int kMaxSlotValues = 2048;
constexpr int kCtlPieces = 8;         // control ops are split into up to this many warp tasks
// Record chunk: the unit of a warp's record fetches (plan option page_bytes,
// a power of two).
constexpr int kDefaultChunkBytes = 1024;
constexpr int kMinChunkBytes = 512;
constexpr int kMaxChunkBytes = 4096;

}  // namespace sht
