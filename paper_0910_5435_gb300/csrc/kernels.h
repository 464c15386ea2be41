// kernels.h -- host-side launch interface of the CUDA kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sht_stream.h"

namespace sht {

// Arguments of the persistent butterfly sweep (one launch = one direction of
// the Legendre stage for every order m).
// One field of a batched launch: its plan's factor stream (device memory,
// set when the batch is created).
struct FieldDesc {
  const uint8_t* pages;
  const uint8_t* values;
  const double* prescale;      // FOLD prescale or nullptr
  const double2* twiddle;      // per-order phase or nullptr
  int l;
  int pad;
};

struct SweepArgs {
  const uint8_t* pages;        // stream pages (device)
  const uint8_t* values;       // value region (device; ops flagged F_VALUES_APART)
  const UnitEntry* units;      // LPT-ordered unit table (device)
  int n_units;
  int page_bytes;
  int nstages;                 // pages in flight per CTA (TMA ring depth)
  int l;
  int buf_ab;                  // elements of shared vectors A and B
  unsigned long long quit_page;
  const void* in;              // synthesis: beta; analysis: G
  void* out;                   // synthesis: G; analysis: beta
  const double* prescale;      // FOLD: per positive node scale (l entries) or nullptr
  const double2* twiddle;      // per order m: UNFOLD multiplies its outputs, FOLD its inputs (or nullptr)
  unsigned* counter;           // work-queue counter (self-resetting; 0 between launches)
  unsigned* status;            // device status word (0 = ok)
  unsigned long long* trace;   // kTraceSlots cycle counters accumulated over all CTAs, or nullptr
  int num_vecs;                // shared vectors (buffer ids 0 .. num_vecs-1)
  int staged;                  // 1: each consumer warp stages op values in shared slots
  int slot_bytes;              // bytes of one staging slot (staged launches)
  int warp_slots;              // staging slots per consumer warp: 1, or 2 (also for 0)
  // Batched launches (fields != nullptr): units[u].m is the item's field f;
  // pages, values, l, prescale and twiddle come from fields[f], the field's
  // input and output from field_in[f] and field_out[f] (device arrays).
  const FieldDesc* fields;
  const void* const* field_in;
  void* const* field_out;
  int io_align;                // required alignment (bytes) of field_in / field_out entries
};

// Launch shape of a sweep: consumer warps, ring depth, resident CTAs per
// SM, dynamic shared memory, and whether op values are staged per warp.
struct SweepConfig {
  int nw = 8;
  int nstages = 0;
  int ctas_per_sm = 0;
  size_t smem = 0;
  bool staged = false;
  int slot_bytes = 0;
  int warp_slots = 2;
};

// Trace slots (clock64 cycles summed over CTAs): consumer warps executing ops,
// waiting for an op to be published, waiting for its dependencies, waiting
// for staged values; producer waiting for a free page; parser waiting for a
// landed page; ops executed; execution split by op class.
enum TraceSlot {
  TR_EXEC = 0, TR_WAIT_READY, TR_WAIT_DEP, TR_PROD_WAIT, TR_PARSE_WAIT, TR_OPS, TR_WAIT_VALUES,
  TR_EXEC_GEMV,    // cycles in compute ops (part of TR_EXEC)
  TR_EXEC_CTL,     // cycles in control ops (part of TR_EXEC)
  TR_COMPLETE,     // cycles marking ops done (part of TR_EXEC)
  TR_N_GEMV,       // compute ops executed
  TR_N_CTL,        // control ops executed
  kTraceSlots = 16
};

// Kernel precisions: the three stream formats, plus split float32 factors
// applied with float64 accumulation (same streams as PREC_SPLIT32).
enum SweepPrec { PREC_FP64 = 0, PREC_FP32 = 1, PREC_SPLIT32 = 2, PREC_SPLIT32_ACC64 = 3 };

size_t sweep_smem_bytes(int prec, int page_bytes, int nstages, int buf_ab, int num_vecs, int nw, int slot_bytes,
                        int warp_slots = 2);
// Picks the ring depth (nstages > 0: exactly that depth) for the given warps:
// two resident CTAs per SM with at least three pages in flight each if they
// fit, else one CTA with the deepest ring that fits in optin bytes.  Values
// are staged in two slots of slot_bytes per warp (0: values inline) when the
// slots fit beside a ring of two pages.  False if nothing fits.
bool sweep_choose(int prec, int page_bytes, int buf_ab, int num_vecs, int nw, int slot_bytes, int nstages,
                  size_t optin, SweepConfig* c, int warp_slots = 2);
cudaError_t sweep_configure(int prec, size_t smem);
// resident CTAs per SM for this shared-memory size (>= 1); nw = consumer warps (8 or 16)
int sweep_blocks_per_sm(int prec, int nw, size_t smem);
cudaError_t sweep_launch(int prec, int nw, const SweepArgs& a, int grid, size_t smem, cudaStream_t st);

// Direct float64 baseline: dense P-bar blocks, [j][i] per (m, p), i fastest.
struct DirectArgs {
  const double* dense;         // all blocks
  const long long* off;        // [2l * 2] offsets (doubles) of block (m, p)
  const int* rows;             // [2l * 2] kept rows
  const int* ncol;             // [2l * 2] columns n_{m,p}
  const double* w_pos;         // l positive-node weights
  int l;
  const void* in;
  void* out;
};
cudaError_t direct_synth_launch(const DirectArgs& a, cudaStream_t st);
// dst[m][i] = src[m][i] * tw[m] on a [2l][2l] complex array (src == dst allowed)
cudaError_t phase_launch(bool fp32, const void* src, void* dst, const double2* tw, int l, int num_sms,
                         cudaStream_t st);
cudaError_t direct_analysis_launch(const DirectArgs& a, cudaStream_t st);

}  // namespace sht
