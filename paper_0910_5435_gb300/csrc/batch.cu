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

// One launch of a direction: the field groups of one size class (1, 2 or up
// to 4 fields sharing a plan), their item table (LPT over all groups) and
// their field lists.
struct SubLaunch {
  sht::FieldDesc* d_fields = nullptr;
  int* d_group_fields = nullptr;
  sht::UnitEntry* d_units = nullptr;
  int n_units = 0;
  int n_groups = 0;
  int capacity = 1;  // max over groups of nf * buf_ab (elements of each shared vector)
  sht::SweepConfig cfg;
};

constexpr int kClasses = 3;  // groups of 1, 2, and 3 or 4 fields
inline int class_fg(int c) { return c == 0 ? 1 : c == 1 ? 2 : 4; }
inline int class_of(int nf) { return nf <= 1 ? 0 : nf == 2 ? 1 : 2; }

struct BatchDir {
  SubLaunch sub[kClasses];
  int slot_bytes = 0;  // largest staging slot of the fields
  int nw = 16;
  int fcap = 4;        // most fields per group
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

void free_dir(BatchDir& D);

void free_batch(sht_batch_t b) {
  if (!b) return;
  for (BatchDir& d : b->dir) free_dir(d);
  cudaFree(b->d_scratch);
  cudaFree(b->d_tables);
  cudaFreeHost(b->h_stage);
  for (cudaEvent_t& e : b->ring_ev)
    if (e) cudaEventDestroy(e);
  delete b;
}

constexpr int kDirs = 5;

// Groups the fields that share a plan (in order of first appearance), as
// many per group as fit the shared vectors of one CTA next to its warps'
// record chunks and staging slots (at most 4; the groups of one plan are of
// balanced sizes), and lays out one launch per group size class.
void free_dir(BatchDir& D) {
  for (SubLaunch& u : D.sub) {
    cudaFree(u.d_fields);
    cudaFree(u.d_group_fields);
    cudaFree(u.d_units);
    u = SubLaunch();
  }
}

// Builds direction d with at most fcap fields per group (1, 2 or 4).
sht_status build_dir(sht_batch_t b, int d, int nfields, const sht_plan_t* plans, sht_precision prec, int fcap) {
  int optin = 0;
  const size_t csize = (b->q == sht::PREC_FP32) ? 8 : 16;  // one complex of the shared vectors
  {
    BatchDir& D = b->dir[d];
    free_dir(D);
    D.fcap = fcap;
    // the adjoint runs the analysis stream with the 1/w fold prescale; the
    // grid directions run the synthesis and analysis streams with the phase
    const int stream_dir = (d == 0 || d == 3) ? 0 : 1;
    std::vector<sht_plan_t> order;
    std::vector<std::vector<int>> members;
    std::vector<sht::StreamView> views;
    for (int f = 0; f < nfields; ++f) {
      size_t k = 0;
      while (k < order.size() && order[k] != plans[f]) ++k;
      if (k == order.size()) {
        sht::StreamView v;
        const sht_status s = sht::stream_view(plans[f], prec, stream_dir, &v);
        if (s != SHT_OK) return s;
        if (order.empty()) {
          b->device = v.device;
          b->num_sms = v.num_sms;
          b->page_bytes = v.page_bytes;
          D.nw = v.consumer_warps;
        } else if (v.device != b->device || v.page_bytes != b->page_bytes || v.consumer_warps != D.nw) {
          // one launch runs every field's items on the same warps and chunk ring
          sht::set_error_detail("sht_batch_create", "plans differ in device, page_bytes or consumer_warps");
          return SHT_ERR_INVALID_ARG;
        }
        D.slot_bytes = std::max(D.slot_bytes, v.slot_bytes);
        order.push_back(plans[f]);
        members.emplace_back();
        views.push_back(v);
      }
      members[k].push_back(f);
    }
    if (optin == 0) {
      BCK(cudaSetDevice(b->device));
      BCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    }
    // shared-vector capacity (elements of each of A and B) left beside the warps
    const size_t fixed = sht::sweep_smem_bytes(b->q, b->page_bytes, 0, 2, D.nw, D.slot_bytes, 1);
    const size_t cap_max = (size_t)optin > fixed + 128 ? ((size_t)optin - fixed - 128) / (2 * csize) : 0;
    std::vector<sht::FieldDesc> gdesc[kClasses];
    std::vector<int> gfields[kClasses];
    std::vector<sht::UnitEntry> units[kClasses];
    for (size_t k = 0; k < order.size(); ++k) {
      const sht::StreamView& v = views[k];
      const int n = (int)members[k].size();
      int F = 1;
      if (D.nw == 16 && v.buf_ab > 0)
        F = (int)std::min<size_t>((size_t)fcap, std::max<size_t>(1, cap_max / (size_t)v.buf_ab));
      F = std::min(F, n);
      const int ng = (n + F - 1) / F;
      for (int g = 0, at = 0; g < ng; ++g) {
        const int nf = n / ng + (g < n % ng ? 1 : 0);  // balanced group sizes
        const int c = class_of(nf);
        sht::FieldDesc fd{};
        fd.pages = v.pages;
        fd.values = v.values;
        fd.prescale = d == 2 ? v.prescale : nullptr;
        fd.twiddle = d == 3 ? v.tw_syn : d == 4 ? v.tw_ana : nullptr;
        fd.l = v.l;
        fd.buf_ab = v.buf_ab;
        fd.f0 = (int)gfields[c].size();
        fd.nf = nf;
        for (int j = 0; j < nf; ++j) gfields[c].push_back(members[k][at + j]);
        at += nf;
        const uint32_t gi = (uint32_t)gdesc[c].size();
        gdesc[c].push_back(fd);
        for (int u = 0; u < v.n_units; ++u) {
          sht::UnitEntry e = v.units[u];
          e.m = gi;
          units[c].push_back(e);
        }
        D.sub[c].capacity = std::max(D.sub[c].capacity, nf * v.buf_ab);
      }
    }
    for (int c = 0; c < kClasses; ++c) {
      SubLaunch& U = D.sub[c];
      if (gdesc[c].empty()) continue;
      std::stable_sort(units[c].begin(), units[c].end(),
                       [](const sht::UnitEntry& x, const sht::UnitEntry& y) { return x.len16 > y.len16; });
      U.n_units = (int)units[c].size();
      U.n_groups = (int)gdesc[c].size();
      BCK(cudaMalloc(&U.d_fields, sizeof(sht::FieldDesc) * gdesc[c].size()));
      BCK(cudaMalloc(&U.d_group_fields, sizeof(int) * gfields[c].size()));
      BCK(cudaMalloc(&U.d_units, sizeof(sht::UnitEntry) * std::max<size_t>(1, units[c].size())));
      BCK(cudaMemcpy(U.d_fields, gdesc[c].data(), sizeof(sht::FieldDesc) * gdesc[c].size(), cudaMemcpyHostToDevice));
      BCK(cudaMemcpy(U.d_group_fields, gfields[c].data(), sizeof(int) * gfields[c].size(), cudaMemcpyHostToDevice));
      BCK(cudaMemcpy(U.d_units, units[c].data(), sizeof(sht::UnitEntry) * units[c].size(), cudaMemcpyHostToDevice));
    }
    b->optin = (size_t)optin;
    BCK(sht::sweep_configure(b->q, b->optin));
    for (SubLaunch& U : D.sub)
      if (U.n_groups && !sht::sweep_choose(b->q, b->page_bytes, U.capacity, 2, D.nw, D.slot_bytes, 1, b->optin, &U.cfg))
        return SHT_ERR_UNSUPPORTED;
  }
  return SHT_OK;
}

sht_status build(sht_batch_t b, int nfields, const sht_plan_t* plans, sht_precision prec) {
  for (int d = 0; d < kDirs; ++d) {
    const sht_status s = build_dir(b, d, nfields, plans, prec, 4);
    if (s != SHT_OK) return s;
  }
  BCK(cudaMalloc(&b->d_scratch, sizeof(unsigned) * (kDirs * kClasses + 1)));
  BCK(cudaMemset(b->d_scratch, 0, sizeof(unsigned) * (kDirs * kClasses + 1)));
  b->plans.assign(plans, plans + nfields);
  BCK(cudaMalloc(&b->d_tables, sizeof(void*) * kRing * 2 * nfields));
  BCK(cudaMallocHost(&b->h_stage, sizeof(void*) * kRing * 2 * nfields));
  for (cudaEvent_t& e : b->ring_ev) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return SHT_OK;
}

// The launches of direction d, one per non-empty group size class, in order
// on stream.
sht_status launch(sht_batch_t b, int d, const void* const* in, void* const* out, sht_stream_t stream) {
  if (!b || !in || !out) return SHT_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % alignof(void*)) return SHT_ERR_INVALID_ARG;
  const BatchDir& D = b->dir[d];
  BCK(cudaSetDevice(b->device));
  for (int c = 0; c < kClasses; ++c) {
    const SubLaunch& U = D.sub[c];
    if (!U.n_groups) continue;
    sht::SweepArgs a{};
    a.units = U.d_units;
    a.n_units = U.n_units;
    a.chunk_bytes = b->page_bytes;
    a.buf_ab = U.capacity;
    a.counter = b->d_scratch + d * kClasses + c;
    a.status = b->d_scratch + kDirs * kClasses;
    a.num_vecs = 2;
    a.slot_bytes = U.cfg.slot_bytes;
    a.warp_slots = 1;
    a.fields = U.d_fields;
    a.group_fields = U.d_group_fields;
    a.field_in = in;
    a.field_out = out;
    a.io_align = (b->q == sht::PREC_FP32) ? 8 : 16;
    a.fg = class_fg(c);
    const int grid = std::max(1, std::min(b->num_sms * U.cfg.ctas_per_sm, U.n_units));
    (void)cudaGetLastError();
    BCK(sht::sweep_launch(b->q, D.nw, a, grid, U.cfg.smem, reinterpret_cast<cudaStream_t>(stream)));
  }
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
  BCK(cudaMemcpy(&st, b->d_scratch + kDirs * kClasses, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st != 0) {
    // a launch stopped early: its queue counters may not have been reset
    BCK(cudaMemset(b->d_scratch, 0, sizeof(unsigned) * (kDirs * kClasses + 1)));
    return (sht_status)st;
  }
  return SHT_OK;
}

sht_status sht_batch_autotune(sht_batch_t b, int direction, const void* const* in, void* const* out, int reps,
                              sht_stream_t stream) {
  if (!b || direction < 0 || direction >= kDirs || reps < 1) return SHT_ERR_INVALID_ARG;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  BCK(cudaSetDevice(b->device));
  // The plans' work items are scheduled for their consumer warps, which fixes
  // the warps and the shared-memory layout of a launch; what is tuned is how
  // many fields of one plan share a launch's reading of its factor stream
  // (at most 1, 2 or 4 per group, as far as their vectors fit).
  int best_cap = b->dir[direction].fcap;
  float best_ms = -1.f;
  sht_status result = SHT_OK;
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  for (int fcap : {1, 2, 4}) {
    result = build_dir(b, direction, b->n, b->plans.data(), b->prec, fcap);
    if (result != SHT_OK) break;
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
      best_cap = fcap;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const sht_status rebuilt = build_dir(b, direction, b->n, b->plans.data(), b->prec, best_cap);
  return result != SHT_OK ? result : rebuilt;
}

sht_status sht_batch_get_config(sht_batch_t b, int direction, int* consumer_warps, int* nstages, int* ctas_per_sm,
                                int* smem_bytes) {
  if (!b || direction < 0 || direction >= kDirs) return SHT_ERR_INVALID_ARG;
  const BatchDir& D = b->dir[direction];
  int ctas = 0;
  size_t smem = 0;
  for (const SubLaunch& U : D.sub)
    if (U.n_groups) {
      ctas = ctas ? std::min(ctas, U.cfg.ctas_per_sm) : U.cfg.ctas_per_sm;
      smem = std::max(smem, U.cfg.smem);
    }
  if (consumer_warps) *consumer_warps = D.nw;
  if (nstages) *nstages = 2;  // record chunks in flight per warp
  if (ctas_per_sm) *ctas_per_sm = ctas;
  if (smem_bytes) *smem_bytes = (int)smem;
  return SHT_OK;
}

sht_status sht_batch_get_groups(sht_batch_t b, int direction, int* max_fields_per_group, int* groups) {
  if (!b || direction < 0 || direction >= kDirs) return SHT_ERR_INVALID_ARG;
  const BatchDir& D = b->dir[direction];
  int mx = 0, n = 0;
  for (int c = 0; c < kClasses; ++c)
    if (D.sub[c].n_groups) {
      mx = std::max(mx, class_fg(c));
      n += D.sub[c].n_groups;
    }
  if (max_fields_per_group) *max_fields_per_group = mx;
  if (groups) *groups = n;
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
