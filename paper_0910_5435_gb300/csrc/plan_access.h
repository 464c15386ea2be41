// plan_access.h -- internal: the sweep launch of a plan's precision that is
// already on the device, for entry points outside capi.cu.
#pragma once

#include <stddef.h>

#include "../../include/sht.h"
#include "kernels.h"
#include "sht_stream.h"

namespace sht {

struct PreparedSweep {
  SweepArgs args;   // counter, status and trace left null for the caller to set
  int prec = 0;     // SweepPrec of the kernel
  int consumer_warps = 8;
  int slot_bytes = 0;                // staging slot of one warp
  int grid = 1;
  size_t smem = 0;
  int device = 0;
};

// Validates the arguments like the compute entry points and fills *out for a
// precision whose streams are already uploaded.  Builds nothing, uploads
// nothing and allocates nothing: a precision that is not on the device
// yet gives SHT_ERR_UNSUPPORTED.  dir: 0 synthesis, 1 analysis.
sht_status prepared_sweep(sht_plan_t plan, sht_precision prec, int dir, const void* in, void* out,
                          PreparedSweep* out_launch);

// A plan's stream of one precision and direction on the device.
struct StreamView {
  const uint8_t* pages = nullptr;
  const uint8_t* values = nullptr;
  const UnitEntry* units = nullptr;  // host copy of the item table (LPT order)
  int n_units = 0;
  int buf_ab = 0;
  int num_vecs = 2;
  int l = 0;
  int page_bytes = 0;                // record chunk bytes
  int device = 0;
  int num_sms = 0;
  int consumer_warps = 8;
  int slot_bytes = 0;                // staging slot of one warp
  int warp_slots = 1;                // staging slots per consumer warp
  const double* prescale = nullptr;  // 1 / w_{l+i} (adjoint fold)
  const double2* tw_syn = nullptr;   // e^{i pi m / (4l-1)}: the synthesis phase of eq. phis
  const double2* tw_ana = nullptr;   // its conjugate over 4l-1: the analysis phase
};

// Fills *v, building and uploading the precision first if needed (this may
// allocate).  dir: 0 synthesis, 1 analysis.
sht_status stream_view(sht_plan_t plan, sht_precision prec, int dir, StreamView* v);

// The phi stage's FFTs of a plan (cuFFT on stream; the plan's FFT handles are
// made at first use): complex-to-real from the phased [2l][2l] array `in`
// (overwritten) to the [2l][4l-1] grid, and real-to-complex from the grid to
// `out` (before the conjugate phase).
sht_status phi_fft_c2r(sht_plan_t plan, sht_precision prec, void* in, void* values, sht_stream_t stream);
sht_status phi_fft_r2c(sht_plan_t plan, sht_precision prec, const void* values, void* out, sht_stream_t stream);

// Sets the text returned by sht_last_error_detail on this thread.
void set_error_detail(const char* where, const char* what);

}  // namespace sht
