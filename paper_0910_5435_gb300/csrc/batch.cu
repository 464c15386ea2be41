// batch.cu -- many fields, each with its own plan (so its own bandlimit),
// through one persistent sweep launch.
//
// The work items of every field's factor stream go into one item table,
// ordered by decreasing size over all fields (longest-processing-time
// order), so the CTAs of the persistent kernel balance small and large
// fields together.  Each item carries its field index; the kernel finds the
// field's pages, values and bandlimit in a device table built here once,
// and the field's input and output in caller-owned device arrays of
// pointers.  A call therefore copies and allocates nothing, and the launch
// can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <new>
#include <vector>

#include "../../include/sht.h"
#include "kernels.h"
#include "plan_access.h"

namespace {

struct BatchDir {
  sht::FieldDesc* d_fields = nullptr;
  sht::UnitEntry* d_units = nullptr;
  int n_units = 0;
  int buf_ab = 1;
  int num_vecs = 2;
  int slot_bytes = 0;  // largest staging slot of the fields
  sht::SweepConfig cfg;
};

}  // namespace

// Device pointer tables of the grid entry points, filled from host arrays:
// kRing slots, each the input then the output pointers of one call, copied
// from pinned staging on the call's stream.  A slot is reused only after the
// event recorded behind its last launch has completed.
constexpr int kRing = 4;

struct sht_batch_s {
  int n = 0;
  int q = 0;  // sht::SweepPrec
  sht_precision prec = SHT_FP64;
  int device = 0;
  int num_sms = 0;
  int page_bytes = 0;
  size_t optin = 0;
  // synthesis, analysis, adjoint of synthesis; synthesis and analysis with
  // the phase of the phi stage fused (the grid entry points)
  BatchDir dir[5];
  unsigned* d_scratch = nullptr;  // queue counter per direction, then the status word
  std::vector<sht_plan_t> plans;
  void** d_tables = nullptr;  // kRing x 2n device pointers
  void** h_stage = nullptr;   // kRing x 2n, pinned
  cudaEvent_t ring_ev[kRing] = {};
  int ring_next = 0;
};

namespace {

#define BCK(x)                                                          \
  do {                                                                  \
    const cudaError_t e_ = (x);                                         \
    if (e_ != cudaSuccess) {                                            \
      sht::set_error_detail("batch", cudaGetErrorString(e_));           \
      return SHT_ERR_CUDA;                                              \
    }                                                                   \
  } while (0)

void free_batch(sht_batch_t b) {
  if (!b) return;
  for (BatchDir& d : b->dir) {
    cudaFree(d.d_fields);
    cudaFree(d.d_units);
  }
  cudaFree(b->d_scratch);
  cudaFree(b->d_tables);
  cudaFreeHost(b->h_stage);
  for (cudaEvent_t& e : b->ring_ev)
    if (e) cudaEventDestroy(e);
  delete b;
}

constexpr int kDirs = 5;

sht_status build(sht_batch_t b, int nfields, const sht_plan_t* plans, sht_precision prec) {
  for (int d = 0; d < kDirs; ++d) {
    std::vector<sht::FieldDesc> fields(nfields);
    std::vector<sht::UnitEntry> units;
    BatchDir& D = b->dir[d];
    for (int f = 0; f < nfields; ++f) {
      sht::StreamView v;
      // the adjoint runs the analysis stream with the 1/w fold prescale; the
      // grid directions run the synthesis and analysis streams with the phase
      const int stream_dir = (d == 0 || d == 3) ? 0 : 1;
      const sht_status s = sht::stream_view(plans[f], prec, stream_dir, &v);
      if (s != SHT_OK) return s;
      if (f == 0) {
        b->device = v.device;
        b->num_sms = v.num_sms;
        b->page_bytes = v.page_bytes;
        D.cfg.nw = v.consumer_warps;
      } else if (v.device != b->device || v.page_bytes != b->page_bytes || v.consumer_warps != D.cfg.nw) {
        // one launch runs every field's items on the same warps and chunk ring
        sht::set_error_detail("sht_batch_create", "plans differ in device, page_bytes or consumer_warps");
        return SHT_ERR_INVALID_ARG;
      }
      fields[f].pages = v.pages;
      fields[f].values = v.values;
      fields[f].prescale = d == 2 ? v.prescale : nullptr;
      fields[f].twiddle = d == 3 ? v.tw_syn : d == 4 ? v.tw_ana : nullptr;
      fields[f].l = v.l;
      D.buf_ab = std::max(D.buf_ab, v.buf_ab);
      D.num_vecs = std::max(D.num_vecs, v.num_vecs);
      D.slot_bytes = std::max(D.slot_bytes, v.slot_bytes);
      for (int u = 0; u < v.n_units; ++u) {
        sht::UnitEntry e = v.units[u];
        e.m = (uint32_t)f;
        units.push_back(e);
      }
    }
    std::stable_sort(units.begin(), units.end(),
                     [](const sht::UnitEntry& a, const sht::UnitEntry& c) { return a.len16 > c.len16; });
    D.n_units = (int)units.size();
    BCK(cudaSetDevice(b->device));
    BCK(cudaMalloc(&D.d_fields, sizeof(sht::FieldDesc) * fields.size()));
    BCK(cudaMalloc(&D.d_units, sizeof(sht::UnitEntry) * std::max<size_t>(1, units.size())));
    BCK(cudaMemcpy(D.d_fields, fields.data(), sizeof(sht::FieldDesc) * fields.size(), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(D.d_units, units.data(), sizeof(sht::UnitEntry) * units.size(), cudaMemcpyHostToDevice));
  }
  BCK(cudaMalloc(&b->d_scratch, sizeof(unsigned) * (kDirs + 1)));
  BCK(cudaMemset(b->d_scratch, 0, sizeof(unsigned) * (kDirs + 1)));
  b->plans.assign(plans, plans + nfields);
  BCK(cudaMalloc(&b->d_tables, sizeof(void*) * kRing * 2 * nfields));
  BCK(cudaMallocHost(&b->h_stage, sizeof(void*) * kRing * 2 * nfields));
  for (cudaEvent_t& e : b->ring_ev) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  int optin = 0;
  BCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
  b->optin = (size_t)optin;
  BCK(sht::sweep_configure(b->q, b->optin));
  for (BatchDir& D : b->dir)
    if (!sht::sweep_choose(b->q, b->page_bytes, D.buf_ab, D.num_vecs, D.cfg.nw, D.slot_bytes, 1, b->optin, &D.cfg))
      return SHT_ERR_UNSUPPORTED;
  return SHT_OK;
}

sht_status launch(sht_batch_t b, int d, const void* const* in, void* const* out, sht_stream_t stream) {
  if (!b || !in || !out) return SHT_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % alignof(void*)) return SHT_ERR_INVALID_ARG;
  const BatchDir& D = b->dir[d];
  BCK(cudaSetDevice(b->device));
  sht::SweepArgs a{};
  a.units = D.d_units;
  a.n_units = D.n_units;
  a.chunk_bytes = b->page_bytes;
  a.buf_ab = D.buf_ab;
  a.counter = b->d_scratch + d;
  a.status = b->d_scratch + kDirs;
  a.num_vecs = D.num_vecs;
  a.slot_bytes = D.cfg.slot_bytes;
  a.warp_slots = 1;
  a.fields = D.d_fields;
  a.field_in = in;
  a.field_out = out;
  a.io_align = (b->q == sht::PREC_FP32) ? 8 : 16;
  const int grid = std::max(1, std::min(b->num_sms * D.cfg.ctas_per_sm, D.n_units));
  (void)cudaGetLastError();
  BCK(sht::sweep_launch(b->q, D.cfg.nw, a, grid, D.cfg.smem, reinterpret_cast<cudaStream_t>(stream)));
  return SHT_OK;
}

// Copies the host pointer arrays in and out into the next ring slot (on
// stream) and runs direction d with them.
sht_status launch_from_host(sht_batch_t b, int d, const void* const* in, void* const* out, sht_stream_t stream) {
  const size_t al = (b->q == sht::PREC_FP32) ? 8 : 16;
  for (int f = 0; f < b->n; ++f)
    if (!in[f] || !out[f] || reinterpret_cast<uintptr_t>(in[f]) % al || reinterpret_cast<uintptr_t>(out[f]) % al)
      return SHT_ERR_INVALID_ARG;
  const int s = b->ring_next;
  b->ring_next = (s + 1) % kRing;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  BCK(cudaEventSynchronize(b->ring_ev[s]));  // the slot's previous copy and launch are done
  void** h = b->h_stage + (size_t)s * 2 * b->n;
  void** dt = b->d_tables + (size_t)s * 2 * b->n;
  for (int f = 0; f < b->n; ++f) {
    h[f] = const_cast<void*>(in[f]);
    h[b->n + f] = out[f];
  }
  BCK(cudaMemcpyAsync(dt, h, sizeof(void*) * 2 * b->n, cudaMemcpyHostToDevice, st));
  const sht_status r = launch(b, d, dt, dt + b->n, stream);
  BCK(cudaEventRecord(b->ring_ev[s], st));
  return r;
}

}  // namespace

extern "C" {

sht_status sht_batch_create(int nfields, const sht_plan_t* plans, sht_precision prec, sht_batch_t* out) {
  if (!out) return SHT_ERR_INVALID_ARG;
  *out = nullptr;
  if (nfields < 1 || nfields > SHT_BATCH_MAX_FIELDS || !plans) return SHT_ERR_INVALID_ARG;
  if (prec != SHT_FP64 && prec != SHT_FP32 && prec != SHT_SPLIT32 && prec != SHT_SPLIT32_ACC64)
    return SHT_ERR_INVALID_ARG;
  for (int f = 0; f < nfields; ++f)
    if (!plans[f]) return SHT_ERR_INVALID_ARG;
  sht_batch_t b = new (std::nothrow) sht_batch_s();
  if (!b) return SHT_ERR_OOM;
  b->n = nfields;
  b->prec = prec;
  b->q = prec == SHT_FP64      ? sht::PREC_FP64
         : prec == SHT_FP32    ? sht::PREC_FP32
         : prec == SHT_SPLIT32 ? sht::PREC_SPLIT32
                               : sht::PREC_SPLIT32_ACC64;
  const sht_status s = build(b, nfields, plans, prec);
  if (s != SHT_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return SHT_OK;
}

sht_status sht_batch_destroy(sht_batch_t b) {
  if (b) {
    cudaSetDevice(b->device);
    free_batch(b);
  }
  return SHT_OK;
}

sht_status sht_batch_synthesize(sht_batch_t b, const void* const* beta, void* const* G, sht_stream_t stream) {
  return launch(b, 0, beta, G, stream);
}

sht_status sht_batch_analyze(sht_batch_t b, const void* const* G, void* const* beta, sht_stream_t stream) {
  return launch(b, 1, G, beta, stream);
}

sht_status sht_batch_synthesize_adjoint(sht_batch_t b, const void* const* G, void* const* beta,
                                        sht_stream_t stream) {
  return launch(b, 2, G, beta, stream);
}

sht_status sht_batch_synthesize_grid(sht_batch_t b, const void* const* beta, void* const* values,
                                     void* const* workspace, sht_stream_t stream) {
  if (!b || !beta || !values || !workspace) return SHT_ERR_INVALID_ARG;
  const size_t al = (b->q == sht::PREC_FP32) ? 8 : 16;
  for (int f = 0; f < b->n; ++f)
    if (!values[f] || reinterpret_cast<uintptr_t>(values[f]) % al) return SHT_ERR_INVALID_ARG;
  BCK(cudaSetDevice(b->device));
  // one launch: every field's Legendre stage with the phase, into its workspace
  sht_status s = launch_from_host(b, 3, beta, workspace, stream);
  if (s != SHT_OK) return s;
  // then each field's complex-to-real FFTs
  for (int f = 0; f < b->n && s == SHT_OK; ++f) s = sht::phi_fft_c2r(b->plans[f], b->prec, workspace[f], values[f], stream);
  return s;
}

sht_status sht_batch_analyze_grid(sht_batch_t b, const void* const* values, void* const* beta,
                                  void* const* workspace, sht_stream_t stream) {
  if (!b || !beta || !values || !workspace) return SHT_ERR_INVALID_ARG;
  const size_t al = (b->q == sht::PREC_FP32) ? 8 : 16;
  for (int f = 0; f < b->n; ++f)
    if (!values[f] || !workspace[f] || !beta[f] || reinterpret_cast<uintptr_t>(workspace[f]) % al ||
        reinterpret_cast<uintptr_t>(beta[f]) % al || reinterpret_cast<uintptr_t>(values[f]) % al)
      return SHT_ERR_INVALID_ARG;
  BCK(cudaSetDevice(b->device));
  // each field's real-to-complex FFTs into its workspace
  sht_status s = SHT_OK;
  for (int f = 0; f < b->n && s == SHT_OK; ++f) s = sht::phi_fft_r2c(b->plans[f], b->prec, values[f], workspace[f], stream);
  if (s != SHT_OK) return s;
  // then one launch: every field's transposed butterfly with the conjugate phase
  return launch_from_host(b, 4, workspace, beta, stream);
}

sht_status sht_batch_last_device_status(sht_batch_t b, sht_stream_t stream) {
  if (!b) return SHT_ERR_INVALID_ARG;
  BCK(cudaSetDevice(b->device));
  BCK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  unsigned st = 0;
  BCK(cudaMemcpy(&st, b->d_scratch + kDirs, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st != 0) {
    // a launch stopped early: its queue counter may not have been reset
    BCK(cudaMemset(b->d_scratch, 0, sizeof(unsigned) * (kDirs + 1)));
    return (sht_status)st;
  }
  return SHT_OK;
}

sht_status sht_batch_autotune(sht_batch_t b, int direction, const void* const* in, void* const* out, int reps,
                              sht_stream_t stream) {
  if (!b || direction < 0 || direction >= kDirs || reps < 1) return SHT_ERR_INVALID_ARG;
  BatchDir& D = b->dir[direction];
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  BCK(cudaSetDevice(b->device));
  // The plans' work items are scheduled for their consumer warps, which fixes
  // the warps and the shared-memory layout of the launch; what remains to
  // choose is the number of CTAs per SM where more than one fits.
  const sht::SweepConfig keep = D.cfg;
  sht::SweepConfig best = keep;
  float best_ms = -1.f;
  sht_status result = SHT_OK;
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  for (int ctas = 1; ctas <= std::max(1, keep.ctas_per_sm) && result == SHT_OK; ++ctas) {
    D.cfg = keep;
    D.cfg.ctas_per_sm = ctas;
    result = launch(b, direction, in, out, stream);  // warm-up
    if (result != SHT_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && result == SHT_OK; ++r) result = launch(b, direction, in, out, stream);
    cudaEventRecord(e1, st);
    if (result != SHT_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      result = SHT_ERR_CUDA;
      break;
    }
    result = sht_batch_last_device_status(b, stream);
    if (result != SHT_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      best = D.cfg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  D.cfg = (result == SHT_OK) ? best : keep;
  return result;
}

sht_status sht_batch_get_config(sht_batch_t b, int direction, int* consumer_warps, int* nstages, int* ctas_per_sm,
                                int* smem_bytes) {
  if (!b || direction < 0 || direction >= kDirs) return SHT_ERR_INVALID_ARG;
  const sht::SweepConfig& c = b->dir[direction].cfg;
  if (consumer_warps) *consumer_warps = c.nw;
  if (nstages) *nstages = 2;  // record chunks in flight per warp
  if (ctas_per_sm) *ctas_per_sm = c.ctas_per_sm;
  if (smem_bytes) *smem_bytes = (int)c.smem;
  return SHT_OK;
}

// Per-field parts of one workspace buffer: field f starts at the sum of the
// preceding fields' workspace bytes, each rounded up to 256 bytes.
size_t sht_batched_workspace_bytes(int nfields, const sht_plan_t* plans, sht_precision prec) {
  if (nfields < 1 || nfields > SHT_BATCH_MAX_FIELDS || !plans) return 0;
  size_t total = 0;
  for (int f = 0; f < nfields; ++f) {
    if (!plans[f]) return 0;
    total += (sht_workspace_bytes(plans[f], prec) + 255) & ~size_t(255);
  }
  return total;
}

}  // extern "C"

namespace {

// One call of a batched spelling: a batch for this call, the grid entry point
// of direction d (0 synthesis, 1 analysis), a wait for the stream (the batch's
// tables are read by the launch), then the batch is freed.
sht_status batched_call(int d, int nfields, const sht_plan_t* plans, sht_precision prec, const void* const* in,
                        void* const* out, void* workspace, sht_stream_t stream) {
  if (!in || !out || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return SHT_ERR_INVALID_ARG;
  const size_t need = sht_batched_workspace_bytes(nfields, plans, prec);
  if (need == 0) return SHT_ERR_INVALID_ARG;
  std::vector<void*> ws(nfields);
  size_t off = 0;
  for (int f = 0; f < nfields; ++f) {
    ws[f] = static_cast<uint8_t*>(workspace) + off;
    off += (sht_workspace_bytes(plans[f], prec) + 255) & ~size_t(255);
  }
  sht_batch_t b = nullptr;
  sht_status s = sht_batch_create(nfields, plans, prec, &b);
  if (s != SHT_OK) return s;
  s = d == 0 ? sht_batch_synthesize_grid(b, in, out, ws.data(), stream)
             : sht_batch_analyze_grid(b, in, out, ws.data(), stream);
  const cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  sht_batch_destroy(b);
  if (s != SHT_OK) return s;
  if (e != cudaSuccess) {
    sht::set_error_detail("batched call", cudaGetErrorString(e));
    return SHT_ERR_CUDA;
  }
  return SHT_OK;
}

}  // namespace

extern "C" {

sht_status sht_synthesize_batched(int nfields, const sht_plan_t* plans, sht_precision prec, const void* const* beta,
                                  void* const* values, void* workspace, sht_stream_t stream) {
  return batched_call(0, nfields, plans, prec, beta, values, workspace, stream);
}

sht_status sht_analyze_batched(int nfields, const sht_plan_t* plans, sht_precision prec, const void* const* values,
                               void* const* beta, void* workspace, sht_stream_t stream) {
  return batched_call(1, nfields, plans, prec, values, beta, workspace, stream);
}

}  // extern "C"
