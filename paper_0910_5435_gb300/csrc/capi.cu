// capi.cu -- the C ABI of include/sht.h: plan lifecycle, device upload and
// launches.  All arguments are validated on the host before any launch.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <stdexcept>
#include <thread>
#include <vector>

#include "../../include/sht.h"
#include "kernels.h"
#include "plan_access.h"
#include "plan_host.h"

using sht::PlanHost;
using sht::UnitFact;

namespace {

constexpr int kNumPrec = 3;

// Launch kinds that own a work-queue counter: synthesis, analysis, adjoint.
enum { KIND_SYN = 0, KIND_ANA = 1, KIND_ADJ = 2, KIND_COUNT = 3 };
// Counters are kept per sweep kernel variant (sht::SweepPrec), not per stream
// format: SHT_SPLIT32 and SHT_SPLIT32_ACC64 apply the same streams but are
// different precisions, whose launches may overlap.
constexpr int kNumKernels = 4;
static_assert(sht::PREC_SPLIT32_ACC64 < kNumKernels, "one counter row per sweep kernel variant");
constexpr int kStatusWord = kNumKernels * KIND_COUNT;  // after the counters
constexpr size_t kScratchBytes = sizeof(unsigned) * (kStatusWord + 1);

struct DevStream {
  uint8_t* pages = nullptr;
  uint8_t* values = nullptr;
  sht::UnitEntry* units = nullptr;
  size_t bytes = 0;
  int n_units = 0;
  int buf_ab = 0;
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Stream format of a precision (SHT_SPLIT32_ACC64 applies the split streams).
int prec_index(sht_precision p) {
  switch (p) {
    case SHT_FP64: return sht::PREC_FP64;
    case SHT_FP32: return sht::PREC_FP32;
    case SHT_SPLIT32:
    case SHT_SPLIT32_ACC64: return sht::PREC_SPLIT32;
    default: return -1;
  }
}

// Kernel that applies a precision's streams.
int kernel_prec(sht_precision p) {
  return p == SHT_SPLIT32_ACC64 ? sht::PREC_SPLIT32_ACC64 : prec_index(p);
}

}  // namespace

struct sht_plan_s {
  PlanHost H;
  sht_plan_opts opts{};
  bool host_only = false;
  int device = -1;
  int num_sms = 0;
  int consumer_warps[kNumPrec] = {16, 16, 16};
  int slot_bytes[kNumPrec] = {0, 0, 0};
  int warp_slots[kNumPrec] = {1, 1, 1};  // staging slots per consumer warp
  int num_vecs[kNumPrec] = {2, 2, 2};
  int ctas_per_sm[kNumPrec] = {1, 1, 1};
  DevStream dev[kNumPrec][2];
  bool dev_ready[kNumPrec] = {false, false, false};
  // Precision q is built (and, unless host_only, uploaded) with its launch
  // shape chosen.  Stored with release once everything it guards is written,
  // read with acquire by the launch paths that skip the plan's mutex.
  std::atomic<bool> ready[kNumPrec] = {false, false, false};
  size_t smem[kNumPrec] = {0, 0, 0};
  double* d_inv_w = nullptr;   // 1 / w_{l+i}: the adjoint's fold prescale
  double2* d_tw_syn = nullptr; // e^{i pi m / N}, N = 4l - 1 (phi stage, eq. phis)
  double2* d_tw_ana = nullptr; // e^{-i pi m / N} / N
  cufftHandle fft_c2r[2] = {0, 0};  // [0] float64 (Z2D), [1] float32 (C2R)
  cufftHandle fft_r2c[2] = {0, 0};
  bool fft_ready[2] = {false, false};
  double* d_w_pos = nullptr;   // w_{l+i}
  unsigned* d_scratch = nullptr;  // [kNumKernels * KIND_COUNT] queue counters, then the status word
  unsigned long long* d_trace = nullptr;  // sweep cycle counters while tracing is enabled
  // direct baseline
  double* d_dense = nullptr;
  long long* d_dense_off = nullptr;
  int* d_dense_rows = nullptr;
  int* d_dense_ncol = nullptr;
  size_t dense_bytes = 0;
  // single-block (Gauss-Jacobi) plans: the vectors A and B of the
  // level-by-level launches, in global memory
  void* d_gvec = nullptr;
  size_t gvec_bytes = 0;
  sht_plan_stats_t stats{};
  std::mutex mu;
};

namespace {

thread_local char g_err_detail[256] = "";

void set_detail(const char* where, const char* what) {
  snprintf(g_err_detail, sizeof(g_err_detail), "%s: %s", where, what);
}

sht_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SHT_OK;
  set_detail("cuda", cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return SHT_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return SHT_ERR_NO_DEVICE;
  return SHT_ERR_CUDA;
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e__ = (call);                     \
    if (e__ != cudaSuccess) return cuda_status(e__); \
  } while (0)

void free_dev(sht_plan_t P) {
  if (P->host_only) return;
  for (int q = 0; q < kNumPrec; ++q)
    for (int d = 0; d < 2; ++d) {
      cudaFree(P->dev[q][d].pages);
      cudaFree(P->dev[q][d].values);
      cudaFree(P->dev[q][d].units);
      P->dev[q][d] = DevStream();
    }
  cudaFree(P->d_inv_w);
  cudaFree(P->d_w_pos);
  cudaFree(P->d_tw_syn);
  cudaFree(P->d_tw_ana);
  P->d_tw_syn = P->d_tw_ana = nullptr;
  for (int f = 0; f < 2; ++f)
    if (P->fft_ready[f]) {
      cufftDestroy(P->fft_c2r[f]);
      cufftDestroy(P->fft_r2c[f]);
      P->fft_ready[f] = false;
    }
  cudaFree(P->d_scratch);
  cudaFree(P->d_trace);
  P->d_trace = nullptr;
  cudaFree(P->d_gvec);
  P->d_gvec = nullptr;
  P->gvec_bytes = 0;
  cudaFree(P->d_dense);
  cudaFree(P->d_dense_off);
  cudaFree(P->d_dense_rows);
  cudaFree(P->d_dense_ncol);
  P->d_inv_w = P->d_w_pos = nullptr;
  P->d_scratch = nullptr;
  P->d_dense = nullptr;
  P->d_dense_off = nullptr;
  P->d_dense_rows = P->d_dense_ncol = nullptr;
}

void fill_stats(sht_plan_t P) {
  const PlanHost& H = P->H;
  sht_plan_stats_t& s = P->stats;
  s.l = H.l;
  s.eps_id = H.eps_id;
  s.leaf_cols = H.leaf_cols;
  s.n_units = H.gj ? 1 : 2 * H.l;
  long long nb = 0, sumk = 0, dense = 0, fv = 0, ib = 0, rows = 0, kept = 0, peak = 0;
  double sumk2 = 0, maxT = 0;
  int kmax = 0, lev = 0, ndir = 0;
  for (const UnitFact& U : H.fact64) {
    dense += (long long)H.l * U.n;
    rows += (U.n > 0) ? H.l : 0;
    kept += (U.n > 0) ? U.rows : 0;
    fv += U.values;
    ib += 2 * U.idx;
    peak = std::max(peak, U.peak_words);
    if (U.n > 0 && U.direct) ++ndir;
    lev = std::max(lev, U.levels);
    for (const auto& b : U.blocks) {
      ++nb;
      sumk += b.k;
      sumk2 += (double)b.k * b.k;
      kmax = std::max(kmax, b.k);
      for (double t : b.T) maxT = std::max(maxT, std::fabs(t));
    }
  }
  s.n_blocks = (int)nb;
  s.k_max = kmax;
  s.k_avg = nb ? (double)sumk / nb : 0.0;
  s.k_sigma = nb ? std::sqrt(std::max(0.0, sumk2 / nb - s.k_avg * s.k_avg)) : 0.0;
  s.max_abs_T = maxT;
  s.max_levels = lev;
  s.n_direct_units = ndir;
  s.rows_total = rows;
  s.rows_kept = kept;
  s.dense_values = dense;
  s.factor_values = fv;
  s.index_bytes = ib;
  s.m_max_words = peak;
  long long fv32 = 0;
  for (const UnitFact& U : H.fact32) fv32 += U.values;
  s.factor_values_fp32 = fv32;
  s.stream_bytes_fp64 = (long long)(H.streams[0][0].bytes.size() + H.streams[0][0].values.size());
  s.stream_bytes_fp32 = (long long)(H.streams[1][0].bytes.size() + H.streams[1][0].values.size());
  s.stream_bytes_split32 = (long long)(H.streams[2][0].bytes.size() + H.streams[2][0].values.size());
  s.t_quad = H.t_quad;
  s.t_comp = H.t_comp;
  s.t_factor = H.t_factor;
  s.t_factor_kernel = H.t_factor_kernel;
  double flops = 0.0;
  for (const UnitFact& U : H.fact64) {
    if (U.direct) continue;
    for (const auto& b : U.blocks) {
      const double h = b.r1 - b.r0, w = b.nin, k = b.k;
      // sum_{i<k} (h-i-1)(w-i-1) in closed form
      const double s1 = k * (k - 1) / 2.0, s2 = (k - 1) * k * (2 * k - 1) / 6.0;
      flops += 4.0 * ((h - 1) * (w - 1) * k - (h - 1 + w - 1) * s1 + s2) + k * k * (w - k);
    }
  }
  s.factor_flops = flops;
  long long swaps = 0;
  for (const UnitFact& U : H.fact64) swaps += U.swaps;
  s.id_swaps = swaps;
  s.smem_bytes = (int)std::max({P->smem[0], P->smem[1], P->smem[2]});
  s.page_bytes = P->H.page_bytes;
}

// Host build of one precision's streams (factorization + record encoding).
sht_status build_host(sht_plan_t P, int q) {
  PlanHost& H = P->H;
  if (H.built[q]) return SHT_OK;
  try {
    const double t0 = now_s();
    const bool fp32 = (q == sht::PREC_FP32);
    if ((fp32 ? H.fact32 : H.fact64).empty()) {
      if (H.gj)
        sht::build_gj_factorization(H, fp32);
      else if (P->opts.device_build)
        sht::build_factorizations_device(H, fp32, P->device);
      else
        sht::build_factorizations(H, fp32);
      H.t_factor += now_s() - t0;
    }
    sht::emit_streams(H, q);
    H.t_comp += now_s() - t0;
  } catch (const std::bad_alloc&) {
    return SHT_ERR_OOM;
  } catch (const sht::DeviceError& e) {
    set_detail("plan build", e.what());
    return SHT_ERR_CUDA;
  } catch (const std::exception& e) {
    set_detail("plan build", e.what());
    return SHT_ERR_INVALID_ARG;
  } catch (...) {
    return SHT_ERR_INVALID_ARG;
  }
  return SHT_OK;
}

sht_status upload_streams(sht_plan_t P, int q) {
  if (P->dev_ready[q]) return SHT_OK;
  const double t0 = now_s();
  CK(cudaSetDevice(P->device));
  int buf_ab = 0, nvecs = 2;
  for (int d = 0; d < 2; ++d) {
    const sht::Stream& S = P->H.streams[q][d];
    nvecs = std::max(nvecs, S.num_vecs);
    DevStream& D = P->dev[q][d];
    D.bytes = S.bytes.size();
    D.n_units = (int)S.units.size();
    D.buf_ab = std::max(S.max_buf_ab, 1);
    buf_ab = std::max(buf_ab, D.buf_ab);
    CK(cudaMalloc(&D.pages, D.bytes));
    if (!S.values.empty()) {
      CK(cudaMalloc(&D.values, S.values.size()));
      CK(cudaMemcpy(D.values, S.values.data(), S.values.size(), cudaMemcpyHostToDevice));
    }
    CK(cudaMalloc(&D.units, sizeof(sht::UnitEntry) * std::max<size_t>(1, S.units.size())));
    CK(cudaMemcpy(D.pages, S.bytes.data(), D.bytes, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(D.units, S.units.data(), sizeof(sht::UnitEntry) * S.units.size(), cudaMemcpyHostToDevice));
  }
  int optin = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device));
  // the limit is a per-kernel setting shared by every plan: raise it to the
  // device maximum once instead of to this plan's size
  CK(sht::sweep_configure(q, (size_t)optin));
  if (q == sht::PREC_SPLIT32) CK(sht::sweep_configure(sht::PREC_SPLIT32_ACC64, (size_t)optin));
  sht::SweepConfig cfg;
  const int slot_bytes = P->H.slot_values_for(q) * (q == sht::PREC_FP32 ? 4 : 8);
  if (P->H.gj) {
    // single-block plans keep their vectors in global memory: one pair for
    // the plan, sized for its widest precision
    const size_t need = (size_t)nvecs * buf_ab * (q == sht::PREC_FP32 ? 8 : 16);
    if (need > P->gvec_bytes) {
      CK(cudaDeviceSynchronize());  // launches of another precision may still use the old pair
      cudaFree(P->d_gvec);
      P->d_gvec = nullptr;
      P->gvec_bytes = 0;
      CK(cudaMalloc(&P->d_gvec, need));
      P->gvec_bytes = need;
    }
  }
  if (!sht::sweep_choose(q, P->H.page_bytes, P->H.gj ? 0 : buf_ab, nvecs, P->consumer_warps[q], slot_bytes, 1,
                         (size_t)optin, &cfg)) {
    set_detail("upload", "the sweep's shared memory (vectors, record chunks, staging slots) exceeds the device limit");
    return SHT_ERR_UNSUPPORTED;
  }
  P->ctas_per_sm[q] = cfg.ctas_per_sm;
  P->smem[q] = cfg.smem;
  P->slot_bytes[q] = cfg.slot_bytes;
  P->num_vecs[q] = nvecs;
  P->dev[q][0].buf_ab = P->dev[q][1].buf_ab = buf_ab;
  P->dev_ready[q] = true;
  P->stats.t_upload += now_s() - t0;
  return SHT_OK;
}

// Uploads precision q; a failure part-way frees what this precision had
// allocated, so a later attempt starts clean.
sht_status upload(sht_plan_t P, int q) {
  const sht_status s = upload_streams(P, q);
  if (s != SHT_OK && !P->dev_ready[q]) {
    for (int d = 0; d < 2; ++d) {
      cudaFree(P->dev[q][d].pages);
      cudaFree(P->dev[q][d].values);
      cudaFree(P->dev[q][d].units);
      P->dev[q][d] = DevStream();
    }
  }
  return s;
}

// Makes precision q ready; cheap once it is (the launch path calls it every
// time), statistics are refreshed only when something was built.
sht_status ensure_prec(sht_plan_t P, int q) {
  if (P->ready[q].load(std::memory_order_acquire)) return SHT_OK;
  std::lock_guard<std::mutex> g(P->mu);
  if (P->ready[q].load(std::memory_order_relaxed)) return SHT_OK;
  sht_status s = build_host(P, q);
  if (s != SHT_OK) return s;
  if (!P->host_only) {
    s = upload(P, q);
    if (s != SHT_OK) return s;
  }
  fill_stats(P);
  P->ready[q].store(true, std::memory_order_release);
  return SHT_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// The order-based entry points refuse a single-block (Gauss-Jacobi) plan.
bool refuse_gj(sht_plan_t P, const char* where) {
  if (!P->H.gj) return false;
  set_detail(where, "a single-block (Gauss-Jacobi) plan: use sht_gj_forward / sht_gj_inverse");
  return true;
}

sht_status launch_sweep(sht_plan_t P, sht_precision prec, int dir, int kind, const void* in, void* out,
                        const double* prescale, sht_stream_t stream, const double2* twiddle = nullptr) {
  if (!P || !in || !out) return SHT_ERR_INVALID_ARG;
  if (refuse_gj(P, "Legendre stage")) return SHT_ERR_UNSUPPORTED;
  const int q = prec_index(prec);
  if (q < 0) return SHT_ERR_INVALID_ARG;
  if (P->host_only) return SHT_ERR_UNSUPPORTED;
  const size_t al = (q == sht::PREC_FP32) ? 8 : 16;
  if (!aligned(in, al) || !aligned(out, al)) return SHT_ERR_INVALID_ARG;
  sht_status s = ensure_prec(P, q);
  if (s != SHT_OK) return s;
  CK(cudaSetDevice(P->device));
  const DevStream& D = P->dev[q][dir];
  sht::SweepArgs a{};  // single-field launch: no field table
  a.pages = D.pages;
  a.values = D.values;
  a.units = D.units;
  a.n_units = D.n_units;
  a.chunk_bytes = P->H.page_bytes;
  a.l = P->H.l;
  a.buf_ab = D.buf_ab;
  a.in = in;
  a.out = out;
  a.prescale = prescale;
  a.twiddle = twiddle;
  a.trace = P->d_trace;
  a.num_vecs = P->num_vecs[q];
  a.slot_bytes = P->slot_bytes[q];
  a.warp_slots = 1;
  a.fg = 1;
  a.counter = P->d_scratch + (kernel_prec(prec) * KIND_COUNT + kind);
  a.status = P->d_scratch + kStatusWord;
  const int grid = std::max(1, std::min(P->num_sms * P->ctas_per_sm[q], D.n_units));
  (void)cudaGetLastError();  // do not report a stale error left by an earlier call (e.g. inside cuFFT)
  CK(sht::sweep_launch(kernel_prec(prec), P->consumer_warps[q], a, grid, P->smem[q],
                       reinterpret_cast<cudaStream_t>(stream)));
  return SHT_OK;
}

}  // namespace

void sht::set_error_detail(const char* where, const char* what) { set_detail(where, what); }

sht_status sht::prepared_sweep(sht_plan_t P, sht_precision prec, int dir, const void* in, void* out,
                               PreparedSweep* L) {
  if (!P || !in || !out || !L || (dir != 0 && dir != 1)) return SHT_ERR_INVALID_ARG;
  const int q = prec_index(prec);
  if (q < 0) return SHT_ERR_INVALID_ARG;
  if (P->host_only || refuse_gj(P, "prepared_sweep")) return SHT_ERR_UNSUPPORTED;
  const size_t al = (q == sht::PREC_FP32) ? 8 : 16;
  if (!aligned(in, al) || !aligned(out, al)) return SHT_ERR_INVALID_ARG;
  if (!P->ready[q].load(std::memory_order_acquire)) {
    set_detail("prepared_sweep", "precision not on the device yet (sht_prepare uploads it)");
    return SHT_ERR_UNSUPPORTED;
  }
  const DevStream& D = P->dev[q][dir];
  sht::SweepArgs& a = L->args;
  a = sht::SweepArgs{};
  a.pages = D.pages;
  a.values = D.values;
  a.units = D.units;
  a.n_units = D.n_units;
  a.chunk_bytes = P->H.page_bytes;
  a.l = P->H.l;
  a.buf_ab = D.buf_ab;
  a.in = in;
  a.out = out;
  a.prescale = nullptr;
  a.twiddle = nullptr;
  a.trace = nullptr;
  a.counter = nullptr;
  a.status = nullptr;
  a.num_vecs = P->num_vecs[q];
  a.slot_bytes = P->slot_bytes[q];
  a.warp_slots = 1;
  a.fg = 1;
  L->prec = kernel_prec(prec);
  L->consumer_warps = P->consumer_warps[q];
  L->grid = std::max(1, std::min(P->num_sms * P->ctas_per_sm[q], D.n_units));
  L->smem = P->smem[q];
  L->device = P->device;
  return SHT_OK;
}

sht_status sht::stream_view(sht_plan_t P, sht_precision prec, int dir, StreamView* v) {
  if (!P || !v || (dir != 0 && dir != 1)) return SHT_ERR_INVALID_ARG;
  const int q = prec_index(prec);
  if (q < 0) return SHT_ERR_INVALID_ARG;
  if (P->host_only || refuse_gj(P, "batch")) return SHT_ERR_UNSUPPORTED;
  sht_status s = ensure_prec(P, q);
  if (s != SHT_OK) return s;
  const DevStream& D = P->dev[q][dir];
  const sht::Stream& S = P->H.streams[q][dir];
  v->pages = D.pages;
  v->values = D.values;
  v->units = S.units.data();
  v->n_units = (int)S.units.size();
  v->buf_ab = D.buf_ab;
  v->num_vecs = P->num_vecs[q];
  v->l = P->H.l;
  v->page_bytes = P->H.page_bytes;
  v->device = P->device;
  v->num_sms = P->num_sms;
  v->consumer_warps = P->consumer_warps[q];
  v->slot_bytes = P->H.slot_values_for(q) * (q == sht::PREC_FP32 ? 4 : 8);
  v->warp_slots = 1;
  v->prescale = P->d_inv_w;
  v->tw_syn = P->d_tw_syn;
  v->tw_ana = P->d_tw_ana;
  return SHT_OK;
}

extern "C" {

const char* sht_last_error_detail(void) { return g_err_detail; }

const char* sht_status_string(sht_status s) {
  switch (s) {
    case SHT_OK: return "SHT_OK";
    case SHT_ERR_INVALID_ARG: return "SHT_ERR_INVALID_ARG";
    case SHT_ERR_OOM: return "SHT_ERR_OOM";
    case SHT_ERR_CUDA: return "SHT_ERR_CUDA";
    case SHT_ERR_PLAN_CORRUPT: return "SHT_ERR_PLAN_CORRUPT";
    case SHT_ERR_TIMEOUT: return "SHT_ERR_TIMEOUT";
    case SHT_ERR_UNSUPPORTED: return "SHT_ERR_UNSUPPORTED";
    case SHT_ERR_NO_DEVICE: return "SHT_ERR_NO_DEVICE";
  }
  return "SHT_ERR_UNKNOWN";
}

sht_status sht_plan_opts_default(sht_plan_opts* o) {
  if (!o) return SHT_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->leaf_cols = 64;
  o->trim_eps = -1.0;
  o->min_band_rows = 32;
  o->host_only = 0;
  o->num_threads = 0;
  o->page_bytes = 0;
  o->eps_fp32 = 0.0;
  o->consumer_warps = 0;
  o->values_inline = 0;
  o->debug_unmet_dependency = 0;
  o->slot_values = 0;
  o->device_build = 0;
  o->device_build_arena_mb = 0;
  o->plan_cache = nullptr;
  o->staging_slots = 0;
  return SHT_OK;
}

sht_status sht_plan_create(int l, double eps_id, sht_plan_t* out) {
  return sht_plan_create_ex(l, eps_id, nullptr, out);
}

namespace {

// Loads the factorizations of a plan file into P when the file was made
// with P's factorization options (true); false when the file does not exist
// or was made with other options.  Throws sht::PlanFileError if the file is
// corrupt.
bool load_plan_file(sht_plan_t P, const std::string& path) {
  sht::PlanFileInfo info;
  if (!sht::read_plan_file_header(path, &info)) return false;
  const PlanHost& H = P->H;
  if (info.l != H.l || info.eps_id != H.eps_id || info.leaf_cols != H.leaf_cols ||
      info.min_band_rows != H.min_band_rows || info.trim_eps != H.trim_eps)
    return false;
  sht::load_factorizations(P->H, path);
  if (!info.has_fp32 || info.eps_fp32 != H.eps_fp32) P->H.fact32.clear();
  return true;
}

sht_status create_plan(int l, double eps_id, const sht_plan_opts* opts, const char* must_load, sht_plan_t* out);

}  // namespace

sht_status sht_plan_create_ex(int l, double eps_id, const sht_plan_opts* opts, sht_plan_t* out) {
  return create_plan(l, eps_id, opts, nullptr, out);
}

sht_status sht_plan_load(const char* path, const sht_plan_opts* opts, sht_plan_t* out) {
  if (!path || !out) return SHT_ERR_INVALID_ARG;
  *out = nullptr;
  sht::PlanFileInfo info;
  try {
    if (!sht::read_plan_file_header(path, &info)) {
      set_detail("sht_plan_load", (std::string("cannot open ") + path).c_str());
      return SHT_ERR_INVALID_ARG;
    }
  } catch (const sht::PlanFileError& e) {
    set_detail("sht_plan_load", e.what());
    return SHT_ERR_PLAN_CORRUPT;
  }
  sht_plan_opts o;
  if (opts) {
    o = *opts;
  } else {
    sht_plan_opts_default(&o);
  }
  // the factorization options are the file's; the rest are the caller's
  o.leaf_cols = info.leaf_cols;
  o.min_band_rows = info.min_band_rows;
  o.trim_eps = info.trim_eps;
  o.eps_fp32 = info.eps_fp32;
  o.plan_cache = nullptr;
  return create_plan(info.l, info.eps_id, &o, path, out);
}

sht_status sht_plan_save(sht_plan_t P, const char* path) {
  if (!P || !path) return SHT_ERR_INVALID_ARG;
  if (refuse_gj(P, "sht_plan_save")) return SHT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(P->mu);
  try {
    sht::save_factorizations(P->H, path);
  } catch (const std::bad_alloc&) {
    return SHT_ERR_OOM;
  } catch (const std::exception& e) {
    set_detail("sht_plan_save", e.what());
    return SHT_ERR_INVALID_ARG;
  }
  return SHT_OK;
}

namespace {

sht_status create_plan(int l, double eps_id, const sht_plan_opts* opts, const char* must_load, sht_plan_t* out) {
  if (!out) return SHT_ERR_INVALID_ARG;
  *out = nullptr;
  sht_plan_opts o;
  if (opts) {
    o = *opts;
  } else {
    sht_plan_opts_default(&o);
  }
  if (o.page_bytes == 0) o.page_bytes = sht::kDefaultChunkBytes;
  if (o.min_band_rows <= 0) o.min_band_rows = std::max(1, o.leaf_cols / 2);
  if (l < 1 || l > 1024 || !(eps_id > 0.0) || !(eps_id < 1.0)) return SHT_ERR_INVALID_ARG;
  if (o.leaf_cols < 2 || o.leaf_cols > 1024) return SHT_ERR_INVALID_ARG;
  if (o.page_bytes < sht::kMinChunkBytes || o.page_bytes > sht::kMaxChunkBytes || (o.page_bytes & (o.page_bytes - 1)))
    return SHT_ERR_INVALID_ARG;
  if (o.values_inline != 0) return SHT_ERR_INVALID_ARG;  // values always travel apart
  if (o.num_threads < 0) return SHT_ERR_INVALID_ARG;
  if (o.device_build != 0 && (o.device_build != 1 || o.host_only)) return SHT_ERR_INVALID_ARG;
  if (o.device_build_arena_mb < 0) return SHT_ERR_INVALID_ARG;
  if (o.staging_slots < 0 || o.staging_slots > 1) return SHT_ERR_INVALID_ARG;
  if (o.consumer_warps != 0 && o.consumer_warps != 8 && o.consumer_warps != 12 && o.consumer_warps != 16)
    return SHT_ERR_INVALID_ARG;
  if (o.slot_values != 0 && (o.slot_values < sht::kMinSlotValues || o.slot_values > sht::kMaxSlotValues ||
                             o.slot_values % 32 != 0))
    return SHT_ERR_INVALID_ARG;

  sht_plan_t P = new (std::nothrow) sht_plan_s();
  if (!P) return SHT_ERR_OOM;
  P->opts = o;
  P->opts.plan_cache = nullptr;  // the caller's string outlives only this call
  P->host_only = o.host_only != 0;
  // one staging slot per warp; 0 = 16 consumer warps for every precision
  // (the work items are scheduled for this many warps)
  for (int q = 0; q < kNumPrec; ++q) {
    P->warp_slots[q] = 1;
    P->consumer_warps[q] = o.consumer_warps ? o.consumer_warps : 16;
  }
  PlanHost& H = P->H;
  H.l = l;
  H.eps_id = eps_id;
  H.eps_fp32 = o.eps_fp32 > 0.0 ? o.eps_fp32 : std::max(eps_id, 1e-7);
  H.trim_eps = o.trim_eps < 0.0 ? eps_id : o.trim_eps;
  H.leaf_cols = o.leaf_cols;
  H.min_band_rows = o.min_band_rows;
  H.num_threads = o.num_threads;
  H.page_bytes = o.page_bytes;
  H.sched_warps = o.consumer_warps ? o.consumer_warps : 16;
  H.debug_unmet_dep = o.debug_unmet_dependency != 0;
  H.slot_values = o.slot_values;
  H.device_arena_bytes = (long long)o.device_build_arena_mb << 20;

  if (!P->host_only) {
    int dev = 0, count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
      delete P;
      return SHT_ERR_NO_DEVICE;
    }
    if (cudaGetDevice(&dev) != cudaSuccess) {
      delete P;
      return SHT_ERR_CUDA;
    }
    P->device = dev;
    cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  try {
    const double t0 = now_s();
    sht::gl_nodes(2 * l, H.x, H.w, H.sin_pos, H.num_threads);
    H.t_quad = now_s() - t0;
  } catch (...) {
    delete P;
    return SHT_ERR_INVALID_ARG;
  }
  // a plan file replaces the factorization (sht_plan_load: it must; a cache
  // file: when it was made with the same options and is intact)
  const char* file = must_load ? must_load : o.plan_cache;
  bool loaded = false;
  if (file) {
    try {
      const double t0 = now_s();
      loaded = load_plan_file(P, file);
      H.t_comp += now_s() - t0;
    } catch (const std::bad_alloc&) {
      delete P;
      return SHT_ERR_OOM;
    } catch (const sht::PlanFileError& e) {
      set_detail(must_load ? "sht_plan_load" : "plan cache (rebuilt)", e.what());
      if (must_load) {
        delete P;
        return SHT_ERR_PLAN_CORRUPT;
      }
    } catch (const std::exception& e) {
      set_detail(must_load ? "sht_plan_load" : "plan cache (rebuilt)", e.what());
      if (must_load) {
        delete P;
        return SHT_ERR_INVALID_ARG;
      }
    }
    if (must_load && !loaded) {
      delete P;
      return SHT_ERR_INVALID_ARG;
    }
  }
  sht_status s = build_host(P, sht::PREC_FP64);
  if (s != SHT_OK) {
    delete P;
    return s;
  }
  if (o.plan_cache && !loaded) {
    try {
      sht::save_factorizations(H, o.plan_cache);
    } catch (const std::exception& e) {
      set_detail("plan cache", e.what());
      delete P;
      return SHT_ERR_INVALID_ARG;
    }
  }
  if (!P->host_only) {
    std::vector<double> invw(l), wpos(l);
    for (int i = 0; i < l; ++i) {
      wpos[i] = H.w[l + i];
      invw[i] = 1.0 / H.w[l + i];
    }
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&P->d_inv_w, sizeof(double) * l);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_w_pos, sizeof(double) * l);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_scratch, kScratchBytes);
    if (e == cudaSuccess) e = cudaMemcpy(P->d_inv_w, invw.data(), sizeof(double) * l, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->d_w_pos, wpos.data(), sizeof(double) * l, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(P->d_scratch, 0, kScratchBytes);
    if (e == cudaSuccess) {
      const int L = 2 * l, N = 4 * l - 1;
      std::vector<double2> ts(L), ta(L);
      for (int m = 0; m < L; ++m) {
        // pi m / N < pi / 2 for m < 2l: no range reduction issue
        const double a = M_PI * (double)m / (double)N;
        ts[m] = make_double2(std::cos(a), std::sin(a));
        ta[m] = make_double2(std::cos(a) / N, -std::sin(a) / N);
      }
      e = cudaMalloc(&P->d_tw_syn, sizeof(double2) * L);
      if (e == cudaSuccess) e = cudaMalloc(&P->d_tw_ana, sizeof(double2) * L);
      if (e == cudaSuccess) e = cudaMemcpy(P->d_tw_syn, ts.data(), sizeof(double2) * L, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(P->d_tw_ana, ta.data(), sizeof(double2) * L, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      free_dev(P);
      delete P;
      return cuda_status(e);
    }
    s = upload(P, sht::PREC_FP64);
    if (s != SHT_OK) {
      free_dev(P);
      delete P;
      return s;
    }
  }
  fill_stats(P);
  P->ready[sht::PREC_FP64].store(true, std::memory_order_release);
  *out = P;
  return SHT_OK;
}

}  // namespace

sht_status sht_plan_destroy(sht_plan_t P) {
  if (!P) return SHT_OK;
  if (!P->host_only && P->device >= 0) cudaSetDevice(P->device);
  free_dev(P);
  delete P;
  return SHT_OK;
}

sht_status sht_plan_get_stats(sht_plan_t P, sht_plan_stats_t* out) {
  if (!P || !out) return SHT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(P->mu);
  *out = P->stats;
  return SHT_OK;
}

sht_status sht_plan_stats(sht_plan_t P, sht_plan_stats_t* out) { return sht_plan_get_stats(P, out); }

sht_status sht_prepare(sht_plan_t P, sht_precision prec) {
  if (!P) return SHT_ERR_INVALID_ARG;
  const int q = prec_index(prec);
  if (q < 0) return SHT_ERR_INVALID_ARG;
  return ensure_prec(P, q);
}

sht_status sht_plan_nodes(sht_plan_t P, double* x, double* w) {
  if (!P || !x || !w) return SHT_ERR_INVALID_ARG;
  if (refuse_gj(P, "sht_plan_nodes")) return SHT_ERR_UNSUPPORTED;
  std::memcpy(x, P->H.x.data(), sizeof(double) * P->H.x.size());
  std::memcpy(w, P->H.w.data(), sizeof(double) * P->H.w.size());
  return SHT_OK;
}

sht_status sht_plan_stream(sht_plan_t P, sht_precision prec, int direction, void* dst, size_t* bytes,
                           size_t* page_bytes_total) {
  if (!P || !bytes || direction < 0 || direction > 1) return SHT_ERR_INVALID_ARG;
  const int q = prec_index(prec);
  if (q < 0) return SHT_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(P->mu);
    sht_status s = build_host(P, q);
    if (s != SHT_OK) return s;
    fill_stats(P);
  }
  const sht::Stream& S = P->H.streams[q][direction];
  const size_t total = S.bytes.size() + S.values.size();
  if (page_bytes_total) *page_bytes_total = S.bytes.size();
  if (!dst) {
    *bytes = total;
    return SHT_OK;
  }
  if (*bytes < total) return SHT_ERR_INVALID_ARG;
  std::memcpy(dst, S.bytes.data(), S.bytes.size());
  if (!S.values.empty()) std::memcpy(static_cast<uint8_t*>(dst) + S.bytes.size(), S.values.data(), S.values.size());
  *bytes = total;
  return SHT_OK;
}

sht_status sht_legendre_synthesize(sht_plan_t P, sht_precision prec, const void* beta, void* G,
                                   sht_stream_t stream) {
  return launch_sweep(P, prec, 0, KIND_SYN, beta, G, nullptr, stream);
}

sht_status sht_legendre_analyze(sht_plan_t P, sht_precision prec, const void* G, void* beta,
                                sht_stream_t stream) {
  return launch_sweep(P, prec, 1, KIND_ANA, G, beta, nullptr, stream);
}

sht_status sht_legendre_synthesize_adjoint(sht_plan_t P, sht_precision prec, const void* G, void* beta,
                                           sht_stream_t stream) {
  if (!P) return SHT_ERR_INVALID_ARG;
  return launch_sweep(P, prec, 1, KIND_ADJ, G, beta, P->d_inv_w, stream);
}

sht_status sht_last_device_status(sht_plan_t P, sht_stream_t stream) {
  if (!P) return SHT_ERR_INVALID_ARG;
  if (P->host_only) return SHT_ERR_UNSUPPORTED;
  CK(cudaSetDevice(P->device));
  CK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  unsigned st = 0;
  CK(cudaMemcpy(&st, P->d_scratch + kStatusWord, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st != 0) {
    // a kernel stopped early: its queue counter may not have been reset
    CK(cudaMemset(P->d_scratch, 0, kScratchBytes));
    return (sht_status)st;
  }
  return SHT_OK;
}

static sht_status ensure_fft(sht_plan_t P, int f) {
  std::lock_guard<std::mutex> g(P->mu);
  if (P->fft_ready[f]) return SHT_OK;
  const int l = P->H.l, L = 2 * l;
  int n = 4 * l - 1;
  int cembed = L, rembed = n;
  // complex side: element (node i, order m) at i + m * 2l, i.e. the [2l][2l] G layout;
  // real side: values[i][j] at i * N + j
  cufftResult r = cufftPlanMany(&P->fft_c2r[f], 1, &n, &cembed, L, 1, &rembed, 1, n, f ? CUFFT_C2R : CUFFT_Z2D, L);
  if (r != CUFFT_SUCCESS) {
    set_detail("cufftPlanMany (complex-to-real)", std::to_string((int)r).c_str());
    return r == CUFFT_ALLOC_FAILED ? SHT_ERR_OOM : SHT_ERR_CUDA;
  }
  r = cufftPlanMany(&P->fft_r2c[f], 1, &n, &rembed, 1, n, &cembed, L, 1, f ? CUFFT_R2C : CUFFT_D2Z, L);
  if (r != CUFFT_SUCCESS) {
    set_detail("cufftPlanMany (real-to-complex)", std::to_string((int)r).c_str());
    cufftDestroy(P->fft_c2r[f]);
    return r == CUFFT_ALLOC_FAILED ? SHT_ERR_OOM : SHT_ERR_CUDA;
  }
  P->fft_ready[f] = true;
  return SHT_OK;
}

static sht_status fft_c2r(sht_plan_t P, int q, void* H, void* values, sht_stream_t stream) {
  const int f = (q == sht::PREC_FP32) ? 1 : 0;
  sht_status s = ensure_fft(P, f);
  if (s != SHT_OK) return s;
  cufftHandle h = P->fft_c2r[f];
  if (cufftSetStream(h, reinterpret_cast<cudaStream_t>(stream)) != CUFFT_SUCCESS) return SHT_ERR_CUDA;
  const cufftResult r = f ? cufftExecC2R(h, reinterpret_cast<cufftComplex*>(H), reinterpret_cast<cufftReal*>(values))
                          : cufftExecZ2D(h, reinterpret_cast<cufftDoubleComplex*>(H),
                                         reinterpret_cast<cufftDoubleReal*>(values));
  if (r != CUFFT_SUCCESS) set_detail("cufftExec (complex-to-real)", std::to_string((int)r).c_str());
  return r == CUFFT_SUCCESS ? SHT_OK : SHT_ERR_CUDA;
}

static sht_status fft_r2c(sht_plan_t P, int q, const void* values, void* H, sht_stream_t stream) {
  const int f = (q == sht::PREC_FP32) ? 1 : 0;
  sht_status s = ensure_fft(P, f);
  if (s != SHT_OK) return s;
  cufftHandle h = P->fft_r2c[f];
  if (cufftSetStream(h, reinterpret_cast<cudaStream_t>(stream)) != CUFFT_SUCCESS) return SHT_ERR_CUDA;
  // cuFFT does not modify the input of an out-of-place real-to-complex transform
  const cufftResult r =
      f ? cufftExecR2C(h, reinterpret_cast<cufftReal*>(const_cast<void*>(values)), reinterpret_cast<cufftComplex*>(H))
        : cufftExecD2Z(h, reinterpret_cast<cufftDoubleReal*>(const_cast<void*>(values)),
                       reinterpret_cast<cufftDoubleComplex*>(H));
  if (r != CUFFT_SUCCESS) set_detail("cufftExec (real-to-complex)", std::to_string((int)r).c_str());
  return r == CUFFT_SUCCESS ? SHT_OK : SHT_ERR_CUDA;
}

static sht_status phi_args_ok(sht_plan_t P, sht_precision prec, const void* a, const void* b, int& q) {
  if (!P || !a || !b) return SHT_ERR_INVALID_ARG;
  q = prec_index(prec);
  if (q < 0) return SHT_ERR_INVALID_ARG;
  if (P->host_only || refuse_gj(P, "phi stage")) return SHT_ERR_UNSUPPORTED;
  const size_t al = (q == sht::PREC_FP32) ? 8 : 16;
  if (!aligned(a, al) || !aligned(b, al)) return SHT_ERR_INVALID_ARG;
  if (cudaSetDevice(P->device) != cudaSuccess) return SHT_ERR_CUDA;
  return SHT_OK;
}

size_t sht_workspace_bytes(sht_plan_t P, sht_precision prec) {
  if (!P) return 0;
  const size_t L = 2 * (size_t)P->H.l;
  return L * L * (prec == SHT_FP32 ? 8 : 16);
}

sht_status sht_phi_synthesize(sht_plan_t P, sht_precision prec, const void* G, void* values, void* workspace,
                              sht_stream_t stream) {
  int q;
  sht_status s = phi_args_ok(P, prec, G, values, q);
  if (s != SHT_OK) return s;
  if (!workspace || !aligned(workspace, 16)) return SHT_ERR_INVALID_ARG;
  (void)cudaGetLastError();
  CK(sht::phase_launch(q == sht::PREC_FP32, G, workspace, P->d_tw_syn, P->H.l, P->num_sms,
                       reinterpret_cast<cudaStream_t>(stream)));
  return fft_c2r(P, q, workspace, values, stream);
}

sht_status sht_phi_analyze(sht_plan_t P, sht_precision prec, const void* values, void* G, sht_stream_t stream) {
  int q;
  sht_status s = phi_args_ok(P, prec, values, G, q);
  if (s != SHT_OK) return s;
  s = fft_r2c(P, q, values, G, stream);
  if (s != SHT_OK) return s;
  (void)cudaGetLastError();
  CK(sht::phase_launch(q == sht::PREC_FP32, G, G, P->d_tw_ana, P->H.l, P->num_sms,
                       reinterpret_cast<cudaStream_t>(stream)));
  return SHT_OK;
}

sht_status sht_synthesize(sht_plan_t P, sht_precision prec, const void* beta, void* values, void* workspace,
                          sht_stream_t stream) {
  int q;
  sht_status s = phi_args_ok(P, prec, beta, values, q);
  if (s != SHT_OK) return s;
  if (!workspace || !aligned(workspace, 16)) return SHT_ERR_INVALID_ARG;
  s = ensure_fft(P, q == sht::PREC_FP32 ? 1 : 0);
  if (s != SHT_OK) return s;
  s = launch_sweep(P, prec, 0, KIND_SYN, beta, workspace, nullptr, stream, P->d_tw_syn);
  if (s != SHT_OK) return s;
  return fft_c2r(P, q, workspace, values, stream);
}

sht_status sht_analyze(sht_plan_t P, sht_precision prec, const void* values, void* beta, void* workspace,
                       sht_stream_t stream) {
  int q;
  sht_status s = phi_args_ok(P, prec, values, beta, q);
  if (s != SHT_OK) return s;
  if (!workspace || !aligned(workspace, 16)) return SHT_ERR_INVALID_ARG;
  s = fft_r2c(P, q, values, workspace, stream);
  if (s != SHT_OK) return s;
  return launch_sweep(P, prec, 1, KIND_ANA, workspace, beta, nullptr, stream, P->d_tw_ana);
}

sht_status sht_trace_enable(sht_plan_t P, int enable) {
  if (!P) return SHT_ERR_INVALID_ARG;
  if (P->host_only) return SHT_ERR_UNSUPPORTED;
  CK(cudaSetDevice(P->device));
  if (enable && !P->d_trace) {
    CK(cudaMalloc(&P->d_trace, sizeof(unsigned long long) * sht::kTraceSlots));
    CK(cudaMemset(P->d_trace, 0, sizeof(unsigned long long) * sht::kTraceSlots));
  } else if (!enable && P->d_trace) {
    CK(cudaDeviceSynchronize());
    cudaFree(P->d_trace);
    P->d_trace = nullptr;
  }
  return SHT_OK;
}

sht_status sht_trace_read(sht_plan_t P, unsigned long long* out, int reset) {
  if (!P || !out) return SHT_ERR_INVALID_ARG;
  if (!P->d_trace) return SHT_ERR_UNSUPPORTED;
  CK(cudaSetDevice(P->device));
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(out, P->d_trace, sizeof(unsigned long long) * sht::kTraceSlots, cudaMemcpyDeviceToHost));
  if (reset) CK(cudaMemset(P->d_trace, 0, sizeof(unsigned long long) * sht::kTraceSlots));
  return SHT_OK;
}

sht_status sht_direct_prepare(sht_plan_t P) {
  if (!P) return SHT_ERR_INVALID_ARG;
  if (P->host_only) return SHT_ERR_UNSUPPORTED;
  if (refuse_gj(P, "sht_direct_prepare")) return SHT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(P->mu);
  if (P->d_dense) return SHT_OK;
  const PlanHost& H = P->H;
  const int l = H.l, NU = 4 * l;
  std::vector<long long> off(NU);
  std::vector<int> rows(NU), ncol(NU);
  long long tot = 0;
  for (int u = 0; u < NU; ++u) {
    off[u] = tot;
    rows[u] = H.fact64[u].rows;
    ncol[u] = H.fact64[u].n;
    tot += (long long)rows[u] * ncol[u];
  }
  CK(cudaSetDevice(P->device));
  CK(cudaMalloc(&P->d_dense, sizeof(double) * std::max<long long>(1, tot)));
  CK(cudaMalloc(&P->d_dense_off, sizeof(long long) * NU));
  CK(cudaMalloc(&P->d_dense_rows, sizeof(int) * NU));
  CK(cudaMalloc(&P->d_dense_ncol, sizeof(int) * NU));
  CK(cudaMemcpy(P->d_dense_off, off.data(), sizeof(long long) * NU, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P->d_dense_rows, rows.data(), sizeof(int) * NU, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P->d_dense_ncol, ncol.data(), sizeof(int) * NU, cudaMemcpyHostToDevice));
  P->dense_bytes = sizeof(double) * (size_t)tot;
  // generate P-bar blocks with the x^2 recurrence (unweighted), in parallel
  std::atomic<int> next(0);
  std::atomic<int> err(0);
  int nt = H.num_threads > 0 ? H.num_threads : (int)std::thread::hardware_concurrency();
  nt = std::max(1, std::min(nt, 64));
  auto worker = [&]() {
    cudaSetDevice(P->device);
    std::vector<double> blk;
    for (;;) {
      const int u = next.fetch_add(1);
      if (u >= NU || err.load()) break;
      const int r = rows[u], n = ncol[u];
      if (r == 0 || n == 0) continue;
      blk.resize((size_t)r * n);
      sht::ColumnStream cs(H, u / 2, u % 2, r);
      for (int j = 0; j < n; ++j) cs.next(blk.data() + (size_t)j * r);
      for (int i = 0; i < r; ++i) {
        const double s = 1.0 / std::sqrt(2.0 * H.w[l + i]);
        for (int j = 0; j < n; ++j) blk[(size_t)j * r + i] *= s;
      }
      if (cudaMemcpy(P->d_dense + off[u], blk.data(), sizeof(double) * blk.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
        err.store(1);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(worker);
  worker();
  for (auto& t : th) t.join();
  if (err.load()) return SHT_ERR_CUDA;
  return SHT_OK;
}

static sht::DirectArgs direct_args(sht_plan_t P, const void* in, void* out) {
  sht::DirectArgs a;
  a.dense = P->d_dense;
  a.off = P->d_dense_off;
  a.rows = P->d_dense_rows;
  a.ncol = P->d_dense_ncol;
  a.w_pos = P->d_w_pos;
  a.l = P->H.l;
  a.in = in;
  a.out = out;
  return a;
}

sht_status sht_direct_synthesize(sht_plan_t P, const void* beta, void* G, sht_stream_t stream) {
  if (!P || !beta || !G) return SHT_ERR_INVALID_ARG;
  if (P->host_only) return SHT_ERR_UNSUPPORTED;
  if (!P->d_dense) return SHT_ERR_INVALID_ARG;
  if (!aligned(beta, 16) || !aligned(G, 16)) return SHT_ERR_INVALID_ARG;
  CK(cudaSetDevice(P->device));
  (void)cudaGetLastError();
  CK(sht::direct_synth_launch(direct_args(P, beta, G), reinterpret_cast<cudaStream_t>(stream)));
  return SHT_OK;
}

sht_status sht_direct_analyze(sht_plan_t P, const void* G, void* beta, sht_stream_t stream) {
  if (!P || !beta || !G) return SHT_ERR_INVALID_ARG;
  if (P->host_only) return SHT_ERR_UNSUPPORTED;
  if (!P->d_dense) return SHT_ERR_INVALID_ARG;
  if (!aligned(beta, 16) || !aligned(G, 16)) return SHT_ERR_INVALID_ARG;
  CK(cudaSetDevice(P->device));
  (void)cudaGetLastError();
  CK(sht::direct_analysis_launch(direct_args(P, G, beta), reinterpret_cast<cudaStream_t>(stream)));
  return SHT_OK;
}

// ------------------------------------------------ single blocks (Section 4)

namespace {

sht_status create_gj_plan(int n, int m, int parity, double eps_id, const sht_plan_opts* opts, sht_plan_t* out) {
  if (!out) return SHT_ERR_INVALID_ARG;
  *out = nullptr;
  sht_plan_opts o;
  if (opts) {
    o = *opts;
  } else {
    sht_plan_opts_default(&o);
  }
  if (o.page_bytes == 0) o.page_bytes = sht::kDefaultChunkBytes;
  if (o.min_band_rows <= 0) o.min_band_rows = std::max(1, o.leaf_cols / 2);
  if (n < 1 || n > SHT_GJ_MAX_N || m < 0 || m > SHT_GJ_MAX_N || (parity != 0 && parity != 1) || !(eps_id > 0.0) ||
      !(eps_id < 1.0))
    return SHT_ERR_INVALID_ARG;
  if (o.leaf_cols < 2 || o.leaf_cols > 1024) return SHT_ERR_INVALID_ARG;
  if (o.page_bytes < sht::kMinChunkBytes || o.page_bytes > sht::kMaxChunkBytes || (o.page_bytes & (o.page_bytes - 1)))
    return SHT_ERR_INVALID_ARG;
  if (o.values_inline != 0 || o.num_threads < 0 || o.device_build != 0 || o.plan_cache != nullptr ||
      o.debug_unmet_dependency != 0 || o.staging_slots < 0 || o.staging_slots > 1)
    return SHT_ERR_INVALID_ARG;
  if (o.consumer_warps != 0 && o.consumer_warps != 8 && o.consumer_warps != 12 && o.consumer_warps != 16)
    return SHT_ERR_INVALID_ARG;
  if (o.slot_values != 0 && (o.slot_values < sht::kMinSlotValues || o.slot_values > sht::kMaxSlotValues ||
                             o.slot_values % 32 != 0))
    return SHT_ERR_INVALID_ARG;
  sht_plan_t P = new (std::nothrow) sht_plan_s();
  if (!P) return SHT_ERR_OOM;
  P->opts = o;
  P->host_only = o.host_only != 0;
  for (int q = 0; q < kNumPrec; ++q) {
    P->warp_slots[q] = 1;
    P->consumer_warps[q] = o.consumer_warps ? o.consumer_warps : 16;
  }
  PlanHost& H = P->H;
  H.gj = true;
  H.gj_m = m;
  H.gj_p = parity;
  H.l = n;
  H.unit_cols = n;
  H.eps_id = eps_id;
  H.eps_fp32 = o.eps_fp32 > 0.0 ? o.eps_fp32 : std::max(eps_id, 1e-7);
  H.trim_eps = 0.0;  // every node of the block is kept
  H.leaf_cols = o.leaf_cols;
  H.min_band_rows = o.min_band_rows;
  H.num_threads = o.num_threads;
  H.page_bytes = o.page_bytes;
  H.sched_warps = o.consumer_warps ? o.consumer_warps : 16;
  H.slot_values = o.slot_values;
  if (!P->host_only) {
    int dev = 0, count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
      delete P;
      return SHT_ERR_NO_DEVICE;
    }
    if (cudaGetDevice(&dev) != cudaSuccess) {
      delete P;
      return SHT_ERR_CUDA;
    }
    P->device = dev;
    cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  try {
    const double t0 = now_s();
    std::vector<double> rho;
    sht::gauss_jacobi_nodes(m, parity, n, H.row_x, H.row_sin, rho);
    H.row_sqw.resize(n);
    for (int i = 0; i < n; ++i) H.row_sqw[i] = std::sqrt(rho[i]);
    H.t_quad = now_s() - t0;
  } catch (const std::bad_alloc&) {
    delete P;
    return SHT_ERR_OOM;
  } catch (...) {
    delete P;
    return SHT_ERR_INVALID_ARG;
  }
  sht_status s = build_host(P, sht::PREC_FP64);
  if (s != SHT_OK) {
    delete P;
    return s;
  }
  if (!P->host_only) {
    cudaError_t e = cudaMalloc(&P->d_scratch, kScratchBytes);
    if (e == cudaSuccess) e = cudaMemset(P->d_scratch, 0, kScratchBytes);
    if (e != cudaSuccess) {
      free_dev(P);
      delete P;
      return cuda_status(e);
    }
    s = upload(P, sht::PREC_FP64);
    if (s != SHT_OK) {
      free_dev(P);
      delete P;
      return s;
    }
  }
  fill_stats(P);
  P->ready[sht::PREC_FP64].store(true, std::memory_order_release);
  *out = P;
  return SHT_OK;
}

// One direction of a single block: one launch per stage of the
// level-by-level stream, in order on the caller's stream.
sht_status launch_gj(sht_plan_t P, sht_precision prec, int dir, const void* in, void* out, sht_stream_t stream) {
  if (!P || !in || !out) return SHT_ERR_INVALID_ARG;
  if (!P->H.gj) {
    set_detail("sht_gj_forward / sht_gj_inverse", "not a single-block plan (sht_gj_plan_create)");
    return SHT_ERR_UNSUPPORTED;
  }
  const int q = prec_index(prec);
  if (q < 0) return SHT_ERR_INVALID_ARG;
  if (P->host_only) return SHT_ERR_UNSUPPORTED;
  const size_t al = (q == sht::PREC_FP32) ? 8 : 16;
  if (!aligned(in, al) || !aligned(out, al)) return SHT_ERR_INVALID_ARG;
  sht_status s = ensure_prec(P, q);
  if (s != SHT_OK) return s;
  CK(cudaSetDevice(P->device));
  const DevStream& D = P->dev[q][dir];
  const std::vector<uint32_t>& stages = P->H.streams[q][dir].stage_begin;
  (void)cudaGetLastError();  // do not report a stale error left by an earlier call
  for (size_t st = 0; st + 1 < stages.size(); ++st) {
    const int n_units = (int)(stages[st + 1] - stages[st]);
    if (n_units == 0) continue;
    sht::SweepArgs a{};
    a.pages = D.pages;
    a.values = D.values;
    a.units = D.units + stages[st];
    a.n_units = n_units;
    a.chunk_bytes = P->H.page_bytes;
    a.l = P->H.l;
    a.buf_ab = D.buf_ab;
    a.in = in;
    a.out = out;
    a.trace = P->d_trace;
    a.num_vecs = P->num_vecs[q];
    a.slot_bytes = P->slot_bytes[q];
    a.warp_slots = 1;
    a.fg = 1;
    a.plain = 1;
    a.gvec = P->d_gvec;
    a.counter = P->d_scratch + (kernel_prec(prec) * KIND_COUNT + (dir ? KIND_ANA : KIND_SYN));
    a.status = P->d_scratch + kStatusWord;
    const int grid = std::max(1, std::min(P->num_sms * P->ctas_per_sm[q], n_units));
    CK(sht::sweep_launch(kernel_prec(prec), P->consumer_warps[q], a, grid, P->smem[q],
                         reinterpret_cast<cudaStream_t>(stream)));
  }
  return SHT_OK;
}

}  // namespace

sht_status sht_gj_plan_create(int n, int m, int parity, double eps_id, const sht_plan_opts* opts, sht_plan_t* out) {
  return create_gj_plan(n, m, parity, eps_id, opts, out);
}

sht_status sht_gj_forward(sht_plan_t P, sht_precision prec, const void* beta, void* alpha, sht_stream_t stream) {
  return launch_gj(P, prec, 0, beta, alpha, stream);
}

sht_status sht_gj_inverse(sht_plan_t P, sht_precision prec, const void* alpha, void* beta, sht_stream_t stream) {
  return launch_gj(P, prec, 1, alpha, beta, stream);
}

sht_status sht_gj_launches(sht_plan_t P, sht_precision prec, int direction, int* launches) {
  if (!P || !launches || direction < 0 || direction > 1) return SHT_ERR_INVALID_ARG;
  if (!P->H.gj) return SHT_ERR_UNSUPPORTED;
  const int q = prec_index(prec);
  if (q < 0) return SHT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(P->mu);
  sht_status s = build_host(P, q);
  if (s != SHT_OK) return s;
  const std::vector<uint32_t>& st = P->H.streams[q][direction].stage_begin;
  int c = 0;
  for (size_t i = 0; i + 1 < st.size(); ++i) c += st[i + 1] > st[i];
  *launches = c;
  return SHT_OK;
}

}  // extern "C"

// Outside the C ABI block: internal entry points for batch.cu.
sht_status sht::phi_fft_c2r(sht_plan_t P, sht_precision prec, void* in, void* values, sht_stream_t stream) {
  int q;
  sht_status s = phi_args_ok(P, prec, in, values, q);
  if (s != SHT_OK) return s;
  return fft_c2r(P, q, in, values, stream);
}

sht_status sht::phi_fft_r2c(sht_plan_t P, sht_precision prec, const void* values, void* out, sht_stream_t stream) {
  int q;
  sht_status s = phi_args_ok(P, prec, values, out, q);
  if (s != SHT_OK) return s;
  return fft_r2c(P, q, values, out, stream);
}

