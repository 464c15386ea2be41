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
// One field group of a batched launch: its plan's factor stream (device
// memory, set when the batch is created) and the nf fields it applies it to
// (group_fields[f0 .. f0 + nf), indices into the launch's pointer arrays).
struct FieldDesc {
  const uint8_t* pages;
  const uint8_t* values;
  const double* prescale;      // FOLD prescale or nullptr
  const double2* twiddle;      // per-order phase or nullptr
  int l;
  int buf_ab;                  // elements of each field's shared vectors A and B
  int f0;
  int nf;
};

struct SweepArgs {
  const uint8_t* pages;        // record region: the scheduled work items (device)
  const uint8_t* values;       // value region (device)
  const UnitEntry* units;      // LPT-ordered item table (device)
  int n_units;
  int chunk_bytes;             // bytes of one record chunk (a warp's ring holds two)
  int l;
  int buf_ab;                  // elements of shared vectors A and B
  const void* in;              // synthesis: beta; analysis: G
  void* out;                   // synthesis: G; analysis: beta
  const double* prescale;      // FOLD: per positive node scale (l entries) or nullptr
  const double2* twiddle;      // per order m: UNFOLD multiplies its outputs, FOLD its inputs (or nullptr)
  unsigned* counter;           // work-queue counter (self-resetting; 0 between launches)
  unsigned* status;            // device status word (0 = ok)
  unsigned long long* trace;   // kTraceSlots cycle counters accumulated over all CTAs, or nullptr
  int num_vecs;                // shared vectors (buffer ids 0 .. num_vecs-1)
  int slot_bytes;              // bytes of one value staging slot
  int warp_slots;              // staging slots per consumer warp: 1 or 2
  // Batched launches (fields != nullptr): units[u].m is the item's field
  // group g; pages, values, l, prescale, twiddle and the group's fields come
  // from fields[g], each field k's input and output from field_in[k] and
  // field_out[k] (device arrays).  buf_ab is then the launch's capacity:
  // nf * buf_ab of every group fits in it.
  const FieldDesc* fields;
  const int* group_fields;
  const void* const* field_in;
  void* const* field_out;
  int io_align;                // required alignment (bytes) of field_in / field_out entries
  int fg;                      // fields per group the kernel handles (1; batched launches 1, 2 or 4)
  // Single-block transforms (the Gauss-Jacobi form, eqs. transform and
  // transform2): plain != 0 makes GATHER / SCATTER read and write element j
  // of a plain vector (no coefficient triangle, no parity interleave), FOLD
  // read node value r as is, and DENSE_G / GZERO write node value i (no
  // parity unfold, no order row).  gvec != nullptr holds the vectors A and B
  // (num_vecs * buf_ab elements) in global memory, shared by all CTAs of the
  // launch, instead of in shared memory; the launch is then one stage of a
  // level-by-level schedule (no two ops of a launch touch the same element).
  // In plain mode an op's a1 carries the bits of its vector positions io and
  // oo above 16 (the levels of a large block are wider than 65535).
  int plain;
  void* gvec;
};

// Launch shape of a sweep: consumer warps (the warps the streams were
// scheduled for), resident CTAs per SM, dynamic shared memory, value
// staging slots per warp and their size.
struct SweepConfig {
  int nw = 16;
  int ctas_per_sm = 0;
  size_t smem = 0;
  int slot_bytes = 0;
  int warp_slots = 1;
};

// Trace slots (clock64 cycles summed over CTAs and warps): executing compute
// ops, executing control ops, waiting for other warps' ops (dependencies),
// waiting for staged values, waiting for record chunks, waiting at the item
// barrier; then counts of compute and control ops, items, and the cycles of
// publishing completions.
enum TraceSlot {
  TR_EXEC_GEMV = 0, TR_EXEC_CTL, TR_WAIT_DEP, TR_WAIT_VALUES, TR_WAIT_RECORDS, TR_WAIT_BARRIER,
  TR_N_GEMV, TR_N_CTL, TR_N_ITEMS, TR_COMPLETE,
  kTraceSlots = 16
};

// Kernel precisions: the three stream formats, plus split float32 factors
// applied with float64 accumulation (same streams as PREC_SPLIT32).
enum SweepPrec { PREC_FP64 = 0, PREC_FP32 = 1, PREC_SPLIT32 = 2, PREC_SPLIT32_ACC64 = 3 };

size_t sweep_smem_bytes(int prec, int chunk_bytes, int buf_ab, int num_vecs, int nw, int slot_bytes, int warp_slots);
// Fills *c for nw consumer warps (8, 12 or 16), warp_slots staging slots of
// slot_bytes per warp and two record chunks per warp: false if that does not
// fit in optin bytes of shared memory.
bool sweep_choose(int prec, int chunk_bytes, int buf_ab, int num_vecs, int nw, int slot_bytes, int warp_slots,
                  size_t optin, SweepConfig* c);
cudaError_t sweep_configure(int prec, size_t smem);
// resident CTAs per SM for this shared-memory size (>= 1); nw = consumer warps
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
