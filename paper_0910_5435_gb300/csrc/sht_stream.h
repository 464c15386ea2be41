// sht_stream.h -- device layout of the butterfly factor streams.
//
// Shared by the host-side emitter (plan_build.cpp) and the sweep kernels
// (sweep.cu).  One stream exists per (precision, direction); direction 0 is
// synthesis (coefficients -> node values), 1 is analysis (the transposed
// application, Section 2.2 remark after Figure multi).
//
// A stream is a sequence of fixed-size PAGES (page_bytes each, the unit of
// one TMA bulk copy).  Each order m ("unit") owns a contiguous run of pages;
// the unit table lists them in decreasing cost (LPT order for the persistent
// kernel's work queue).  A page holds a sequence of OPS, each 16-byte aligned:
//
//   [OpHdr 32 B][uint16 index lists, padded to 16 B][values, padded to 16 B]
//
// and ends at the first header with bytes == 0 (or at the page end).  Every
// op applies one small dense matrix V ([K][M] layout, M fastest, so the
// threads of a warp that own consecutive outputs o read consecutive values)
// to a vector held in shared memory:
//
//   SYN_INTERP  out[oo + o] = in[io + skel[o]] + sum_s V[s][o] in[io + red[s]]
//               (with F_ACCUM: out[oo + o] += ...; the skel term only for o < nskel)
//               -- one interpolation matrix of an ID (Section 2.1 eq. 2.1,
//               Section 2.2 eqs. 1-6: y = z[skel] + T z[red]);
//   DENSE       out[oo + o] (= or +=) sum_s V[s][o] in[io + s]
//               -- a stored skeleton-column block (the unprocessed blocks of
//               Section 3) or a dense block;
//   ANA_INTERP  out[oo + red[o]] += sum_s V[s][o] in[io + s], and, with F_SKEL,
//               out[oo + skel[t]] += in[io + t]
//               -- the transpose of an interpolation matrix (anterpolation).
//
// Control ops carry no values: GATHER / SCATTER move one parity of beta^m
// between global memory and shared memory, UNFOLD / FOLD apply the parity
// split of Section 2.3 on the symmetric nodes, CLEAR zeroes an accumulator.
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
  OP_GATHER = 1,      // buf[out_buf][oo + j] = beta^m_{m+p+2j}, j < M       (a0 = p, a1 = m)
  OP_SCATTER = 2,     // beta^m_{m+p+2j} = buf[in_buf][io + j], j < M       (a0 = p, a1 = m)
  OP_UNFOLD = 3,      // G[m][l+i] = E_i + O_i, G[m][l-1-i] = E_i - O_i; E = buf2 (M = rows kept
                      //   for p = 0), O = buf3 (K = rows kept for p = 1)    (a1 = m)
  OP_FOLD = 4,        // buf2[i] = s_i (G[m][l+i] + G[m][l-1-i]), buf3[i] = s_i (G[m][l+i] - G[m][l-1-i]),
                      //   i < l, s_i = optional per-node prescale        (a1 = m)
  OP_CLEAR = 5,       // buf[out_buf][oo .. oo + M) = 0
  OP_SYN_INTERP = 6,
  OP_DENSE = 7,
  OP_ANA_INTERP = 8,
};

enum OpFlags : uint8_t {
  F_SYNC_BEFORE = 1,  // all consumer threads synchronize before the op reads its input
  F_ACCUM = 2,        // DENSE / SYN_INTERP: accumulate into the output instead of overwriting it
  F_SKEL = 4,         // ANA_INTERP: also add the skeleton pass-through (nskel entries)
};

struct alignas(16) OpHdr {
  uint32_t bytes;     // size of this op in bytes (multiple of 16); 0 terminates the page
  uint8_t kind;
  uint8_t flags;
  uint8_t in_buf;     // shared-memory vector ids 0..3
  uint8_t out_buf;
  uint16_t M;         // outputs
  uint16_t K;         // inner dimension
  uint16_t nskel;     // SYN_INTERP: M (0 on F_ACCUM chunks); ANA_INTERP with F_SKEL: pass-through inputs
  uint16_t io;        // element offset of the input vector
  uint16_t oo;        // element offset of the output vector
  uint16_t a0;        // parity for GATHER/SCATTER
  uint32_t a1;        // order m for control ops
  uint32_t idx_bytes; // bytes of the index area (padded to 16)
  uint32_t pad;
};
static_assert(sizeof(OpHdr) == 32, "OpHdr must be 32 bytes");

// Index area contents (uint16, offsets relative to io / oo):
//   SYN_INTERP: red[K] then skel[nskel] (nskel = M, or 0 on accumulated chunks)
//   ANA_INTERP: red[M] then (F_SKEL) skel[nskel]
//   others:     none

struct UnitEntry {
  uint64_t first_page;  // index of the unit's first page in the stream
  uint32_t n_pages;
  uint32_t m;
};
static_assert(sizeof(UnitEntry) == 16, "UnitEntry must be 16 bytes");

// Shared-memory vector ids used by the emitter.
enum BufId : uint8_t { BUF_A = 0, BUF_B = 1, BUF_E = 2, BUF_O = 3 };

constexpr int kMaxM = 128;            // outputs per op (4 per lane, 32 lanes)
constexpr int kConsumerWarps = 8;
constexpr int kConsumerThreads = kConsumerWarps * 32;

}  // namespace sht
