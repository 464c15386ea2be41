// sweep.cu -- persistent butterfly sweep kernels (sm_103a).
//
// One launch applies the Legendre stage of every order m in one direction:
// synthesis (Section 2, eq. alternate_expansion, sums over k, through the
// butterfly of Section 2.2 per parity block) or analysis (the transposed
// application, Section 2.2 remark after Figure multi).
//
// Each CTA is persistent: a producer warp pops orders m from an LPT-sorted
// work queue (atomic counter) and streams the order's factor pages from HBM
// into a ring of shared-memory stages with 1-D TMA bulk copies
// (cp.async.bulk + mbarrier complete_tx); eight consumer warps walk the ops
// of each page (see sht_stream.h) on vectors kept in shared memory.  Each op
// is a small GEMV: lanes own consecutive outputs (coalesced, conflict-free
// reads of the [K][M] value block), warps split the inner dimension, and
// partial sums are combined through shared memory after one named barrier.
//
// Every wait is bounded: on timeout the kernel records SHT_ERR_TIMEOUT in the
// device status word, stops issuing copies, waits (bounded) for the copies it
// already issued, and returns.

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "sht_stream.h"

namespace sht {
namespace {

constexpr int kOpQuit = 0xFF;
constexpr long long kTimeoutCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr unsigned kStatusTimeout = 5;              // SHT_ERR_TIMEOUT

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConsumerThreads) : "memory");
}

// Bounded wait on an mbarrier phase; on timeout records the status, raises
// the CTA abort flag and returns false.
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, unsigned* status,
                                             volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > kTimeoutCycles) {
      atomicCAS(status, 0u, kStatusTimeout);
      *abort_flag = 1;
      return false;
    }
  }
}

// ------------------------------------------------------ precision traits

// float64 factors and arithmetic; complex128 I/O.
struct TF64 {
  using V = double;
  using C = double2;
  using IO = double2;
  struct Acc {
    double re, im;
  };
  __device__ static Acc zero() { return {0.0, 0.0}; }
  __device__ static C czero() { return make_double2(0.0, 0.0); }
  __device__ static void fma(Acc& a, V v, const C& x) {
    a.re = __fma_rn(v, x.x, a.re);
    a.im = __fma_rn(v, x.y, a.im);
  }
  __device__ static void add(Acc& a, const C& c) {
    a.re += c.x;
    a.im += c.y;
  }
  __device__ static void merge(Acc& a, const Acc& b) {
    a.re += b.re;
    a.im += b.im;
  }
  __device__ static C to_c(const Acc& a) { return make_double2(a.re, a.im); }
  __device__ static Acc from_c(const C& c) { return {c.x, c.y}; }
  __device__ static C from_io(const IO& v) { return v; }
  __device__ static IO to_io(const C& c) { return c; }
  __device__ static IO io_zero() { return make_double2(0.0, 0.0); }
  __device__ static IO io_add(const IO& a, const IO& b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static IO io_sub(const IO& a, const IO& b) { return make_double2(a.x - b.x, a.y - b.y); }
  __device__ static IO io_scale(const IO& a, double s) { return make_double2(a.x * s, a.y * s); }
  __device__ static IO io_cmul(const IO& a, const double2& t) {
    return make_double2(a.x * t.x - a.y * t.y, a.x * t.y + a.y * t.x);
  }
};

// hi/lo float32 factors, double-float ("compensated") float32 arithmetic;
// complex128 I/O.  Products use the exact FMA split p + e = hi * x_hi and
// the cross terms hi * x_lo + lo * x_hi (lo * x_lo, ~2^-48 relative, is
// dropped); sums use Knuth's TwoSum.  The _rn intrinsics keep the compiler
// from contracting the error-free transformations.
struct TS32 {
  using V = float2;  // {hi, lo}
  using C = float4;  // {re_hi, re_lo, im_hi, im_lo}
  using IO = double2;
  struct Acc {
    float rh, rl, ih, il;
  };
  __device__ static Acc zero() { return {0.f, 0.f, 0.f, 0.f}; }
  __device__ static C czero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static void two_sum_acc(float& sh, float& sl, float p, float e) {
    const float s = __fadd_rn(sh, p);
    const float bb = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
  }
  __device__ static void fma1(float& sh, float& sl, float2 v, float xh, float xl) {
    const float p = __fmul_rn(v.x, xh);
    float e = __fmaf_rn(v.x, xh, -p);
    e = __fmaf_rn(v.x, xl, e);
    e = __fmaf_rn(v.y, xh, e);
    two_sum_acc(sh, sl, p, e);
  }
  __device__ static void fma(Acc& a, V v, const C& x) {
    fma1(a.rh, a.rl, v, x.x, x.y);
    fma1(a.ih, a.il, v, x.z, x.w);
  }
  __device__ static void add(Acc& a, const C& c) {
    two_sum_acc(a.rh, a.rl, c.x, c.y);
    two_sum_acc(a.ih, a.il, c.z, c.w);
  }
  __device__ static void merge(Acc& a, const Acc& b) {
    two_sum_acc(a.rh, a.rl, b.rh, b.rl);
    two_sum_acc(a.ih, a.il, b.ih, b.il);
  }
  __device__ static void renorm(float& h, float& l) {  // fast two-sum, |h| >= |l|
    const float s = __fadd_rn(h, l);
    l = __fsub_rn(l, __fsub_rn(s, h));
    h = s;
  }
  __device__ static C to_c(Acc a) {
    renorm(a.rh, a.rl);
    renorm(a.ih, a.il);
    return make_float4(a.rh, a.rl, a.ih, a.il);
  }
  __device__ static Acc from_c(const C& c) { return {c.x, c.y, c.z, c.w}; }
  __device__ static C from_io(const IO& v) {
    const float rh = __double2float_rn(v.x);
    const float ih = __double2float_rn(v.y);
    return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
  }
  __device__ static IO to_io(const C& c) {
    return make_double2((double)c.x + (double)c.y, (double)c.z + (double)c.w);
  }
  __device__ static IO io_zero() { return make_double2(0.0, 0.0); }
  __device__ static IO io_add(const IO& a, const IO& b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static IO io_sub(const IO& a, const IO& b) { return make_double2(a.x - b.x, a.y - b.y); }
  __device__ static IO io_scale(const IO& a, double s) { return make_double2(a.x * s, a.y * s); }
  __device__ static IO io_cmul(const IO& a, const double2& t) {
    return make_double2(a.x * t.x - a.y * t.y, a.x * t.y + a.y * t.x);
  }
};

// float32 factors and arithmetic; complex64 I/O.
struct TF32 {
  using V = float;
  using C = float2;
  using IO = float2;
  struct Acc {
    float re, im;
  };
  __device__ static Acc zero() { return {0.f, 0.f}; }
  __device__ static C czero() { return make_float2(0.f, 0.f); }
  __device__ static void fma(Acc& a, V v, const C& x) {
    a.re = __fmaf_rn(v, x.x, a.re);
    a.im = __fmaf_rn(v, x.y, a.im);
  }
  __device__ static void add(Acc& a, const C& c) {
    a.re += c.x;
    a.im += c.y;
  }
  __device__ static void merge(Acc& a, const Acc& b) {
    a.re += b.re;
    a.im += b.im;
  }
  __device__ static C to_c(const Acc& a) { return make_float2(a.re, a.im); }
  __device__ static Acc from_c(const C& c) { return {c.x, c.y}; }
  __device__ static C from_io(const IO& v) { return v; }
  __device__ static IO to_io(const C& c) { return c; }
  __device__ static IO io_zero() { return make_float2(0.f, 0.f); }
  __device__ static IO io_add(const IO& a, const IO& b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static IO io_sub(const IO& a, const IO& b) { return make_float2(a.x - b.x, a.y - b.y); }
  __device__ static IO io_scale(const IO& a, double s) {
    return make_float2((float)(a.x * s), (float)(a.y * s));
  }
  __device__ static IO io_cmul(const IO& a, const double2& t) {
    const float tr = (float)t.x, ti = (float)t.y;
    return make_float2(a.x * tr - a.y * ti, a.x * ti + a.y * tr);
  }
};

// ------------------------------------------------------------ ops

template <class TR>
struct Smem {
  using C = typename TR::C;
  C* base;
  int buf_ab, l;
  __device__ C* buf(int id) const {
    return id < 2 ? base + (size_t)id * buf_ab : base + 2 * (size_t)buf_ab + (size_t)(id - 2) * l;
  }
  __device__ C* part(int area) const { return base + 2 * (size_t)buf_ab + 2 * (size_t)l + (size_t)area * kConsumerThreads; }
};

__device__ __forceinline__ size_t tri_off(int m, int L) { return (size_t)m * L - (size_t)m * (m - 1) / 2; }

template <class TR>
__device__ __forceinline__ void run_gemv(const OpHdr& h, const uint8_t* op, const Smem<TR>& S, int area, int ct,
                                         int cw, int lane) {
  using C = typename TR::C;
  using V = typename TR::V;
  using Acc = typename TR::Acc;
  const int M = h.M, K = h.K;
  const uint16_t* idx = reinterpret_cast<const uint16_t*>(op + sizeof(OpHdr));
  const V* val = reinterpret_cast<const V*>(op + sizeof(OpHdr) + h.idx_bytes);
  const C* in = S.buf(h.in_buf) + h.io;
  C* out = S.buf(h.out_buf) + h.oo;
  C* part = S.part(area);
  const bool gather = (h.kind == OP_SYN_INTERP);
  int nsl = kConsumerWarps;
  if (M > 0) {
    const int wo = (M + 31) >> 5;  // 1..4 warps across the outputs
    nsl = kConsumerWarps / wo;     // warps along the inner dimension
    const int o = lane + 32 * (cw % wo);
    const int sl = cw / wo;
    if (sl < nsl && o < M) {
      Acc a0 = TR::zero(), a1 = TR::zero();
      int s = sl;
      for (; s + nsl < K; s += 2 * nsl) {
        const int s1 = s + nsl;
        const int i0 = gather ? (int)idx[s] : s;
        const int i1 = gather ? (int)idx[s1] : s1;
        const V v0 = val[(size_t)s * M + o];
        const V v1 = val[(size_t)s1 * M + o];
        TR::fma(a0, v0, in[i0]);
        TR::fma(a1, v1, in[i1]);
      }
      if (s < K) {
        const int i0 = gather ? (int)idx[s] : s;
        TR::fma(a0, val[(size_t)s * M + o], in[i0]);
      }
      TR::merge(a0, a1);
      part[sl * M + o] = TR::to_c(a0);
    }
  }
  // indices needed after the barrier are read now (the page may be recycled later)
  int sk = -1, ri = -1, pt = -1;
  if (ct < M) {
    if (gather && ct < h.nskel) sk = idx[K + ct];
    if (h.kind == OP_ANA_INTERP) ri = idx[ct];
  }
  if (h.kind == OP_ANA_INTERP && (h.flags & F_SKEL) && ct < h.nskel) pt = idx[M + ct];
  consumer_sync();
  if (ct < M) {
    Acc r = TR::from_c(part[ct]);
    for (int q = 1; q < nsl; ++q) TR::add(r, part[q * M + ct]);
    if (h.kind == OP_ANA_INTERP) {
      TR::add(r, out[ri]);
      out[ri] = TR::to_c(r);
    } else {
      if (sk >= 0) TR::add(r, in[sk]);
      if (h.flags & F_ACCUM) TR::add(r, out[ct]);
      out[ct] = TR::to_c(r);
    }
  }
  if (pt >= 0) {
    Acc r = TR::from_c(out[pt]);
    TR::add(r, in[ct]);
    out[pt] = TR::to_c(r);
  }
}

template <class TR>
__device__ __forceinline__ void run_control(const OpHdr& h, const SweepArgs& A, const Smem<TR>& S, int ct) {
  using C = typename TR::C;
  using IO = typename TR::IO;
  const int l = A.l, L = 2 * l;
  const int m = (int)h.a1;
  switch (h.kind) {
    case OP_GATHER: {
      const IO* beta = reinterpret_cast<const IO*>(A.in) + tri_off(m, L) + h.a0;
      C* dst = S.buf(h.out_buf) + h.oo;
      for (int j = ct; j < h.M; j += kConsumerThreads) dst[j] = TR::from_io(beta[2 * (size_t)j]);
      break;
    }
    case OP_SCATTER: {
      IO* beta = reinterpret_cast<IO*>(A.out) + tri_off(m, L) + h.a0;
      const C* src = S.buf(h.in_buf) + h.io;
      for (int j = ct; j < h.M; j += kConsumerThreads) beta[2 * (size_t)j] = TR::to_io(src[j]);
      break;
    }
    case OP_UNFOLD: {
      IO* G = reinterpret_cast<IO*>(A.out) + (size_t)m * L;
      const C* E = S.buf(BUF_E);
      const C* O = S.buf(BUF_O);
      const double2 tw = A.twiddle ? A.twiddle[m] : make_double2(1.0, 0.0);
      for (int i = ct; i < l; i += kConsumerThreads) {
        const IO e = i < h.M ? TR::to_io(E[i]) : TR::io_zero();
        const IO o = i < h.K ? TR::to_io(O[i]) : TR::io_zero();
        IO gp = TR::io_add(e, o), gm = TR::io_sub(e, o);
        if (A.twiddle) {
          gp = TR::io_cmul(gp, tw);
          gm = TR::io_cmul(gm, tw);
        }
        G[l + i] = gp;
        G[l - 1 - i] = gm;
      }
      break;
    }
    case OP_FOLD: {
      const IO* G = reinterpret_cast<const IO*>(A.in) + (size_t)m * L;
      C* E = S.buf(BUF_E);
      C* O = S.buf(BUF_O);
      const double2 tw = A.twiddle ? A.twiddle[m] : make_double2(1.0, 0.0);
      for (int i = ct; i < l; i += kConsumerThreads) {
        IO gp = G[l + i], gm = G[l - 1 - i];
        if (A.twiddle) {
          gp = TR::io_cmul(gp, tw);
          gm = TR::io_cmul(gm, tw);
        }
        IO e = TR::io_add(gp, gm), o = TR::io_sub(gp, gm);
        if (A.prescale) {
          e = TR::io_scale(e, A.prescale[i]);
          o = TR::io_scale(o, A.prescale[i]);
        }
        E[i] = TR::from_io(e);
        O[i] = TR::from_io(o);
      }
      break;
    }
    case OP_CLEAR: {
      C* dst = S.buf(h.out_buf) + h.oo;
      for (int j = ct; j < h.M; j += kConsumerThreads) dst[j] = TR::czero();
      break;
    }
    default:
      break;
  }
  consumer_sync();
}

__device__ void producer_loop(const SweepArgs& A, uint8_t* stages, uint64_t* full, uint64_t* empty,
                              volatile int* abort_flag) {
  const uint32_t PB = (uint32_t)A.page_bytes;
  const int NST = A.nstages;
  int stage = 0;
  uint32_t phase = 0;
  int issued_phase[16];
  for (int s = 0; s < 16; ++s) issued_phase[s] = -1;
  bool ok = true;
  for (;;) {
    if (*abort_flag) {
      ok = false;
      break;
    }
    const unsigned u = atomicAdd(A.counter, 1u);
    if (u >= (unsigned)A.n_units) {
      // the last CTA to find the queue empty resets it for the next launch
      if (u == (unsigned)A.n_units + gridDim.x - 1) atomicExch(A.counter, 0u);
      break;
    }
    const UnitEntry e = A.units[u];
    for (uint32_t pg = 0; pg < e.n_pages && ok; ++pg) {
      if (!wait_bounded(empty + stage, phase ^ 1u, A.status, abort_flag)) {
        ok = false;
        break;
      }
      mbar_arrive_expect_tx(full + stage, PB);
      bulk_g2s(stages + (size_t)stage * PB, A.pages + (size_t)(e.first_page + pg) * PB, PB, full + stage);
      issued_phase[stage] = (int)phase;
      if (++stage == NST) {
        stage = 0;
        phase ^= 1u;
      }
    }
    if (!ok) break;
  }
  if (ok && wait_bounded(empty + stage, phase ^ 1u, A.status, abort_flag)) {
    mbar_arrive_expect_tx(full + stage, PB);
    bulk_g2s(stages + (size_t)stage * PB, A.pages + (size_t)A.quit_page * PB, PB, full + stage);
    issued_phase[stage] = (int)phase;
  }
  // never leave the CTA with bulk copies still landing in its shared memory
  for (int s = 0; s < NST; ++s)
    if (issued_phase[s] >= 0) wait_bounded(full + s, (uint32_t)issued_phase[s], A.status, abort_flag);
}

template <class TR>
__global__ void __launch_bounds__(kConsumerThreads + 32) bfly_sweep_kernel(const SweepArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NST = A.nstages;
  const size_t PB = (size_t)A.page_bytes;
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * PB);
  uint64_t* empty = full + NST;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NST);
  const size_t vec_off = ((size_t)NST * PB + 16 * (size_t)NST + 16 + 127) & ~size_t(127);
  Smem<TR> S{reinterpret_cast<typename TR::C*>(smem + vec_off), A.buf_ab, A.l};

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kConsumerWarps) {
    if (lane == 0) producer_loop(A, stages, full, empty, abort_flag);
    return;
  }

  // one consumer performs the bounded wait and broadcasts the outcome, so
  // that all consumers leave together if it gives up (none is left waiting
  // in a named barrier)
  volatile int* page_ok = abort_flag + 1;
  int stage = 0, area = 0;
  uint32_t phase = 0;
  for (;;) {
    if (tid == 0) *page_ok = wait_bounded(full + stage, phase, A.status, abort_flag) ? 1 : 0;
    consumer_sync();
    if (!*page_ok) break;
    mbar_try_wait(full + stage, phase);  // completed already: each thread's own acquire of the page
    const uint8_t* page = stages + (size_t)stage * PB;
    bool quit = false;
    for (size_t off = 0; off + sizeof(OpHdr) <= PB;) {
      const OpHdr h = *reinterpret_cast<const OpHdr*>(page + off);
      if (h.bytes == 0) break;
      if (h.kind == kOpQuit) {
        quit = true;
        break;
      }
      if (h.flags & F_SYNC_BEFORE) consumer_sync();
      if (h.kind >= OP_SYN_INTERP) {
        run_gemv<TR>(h, page + off, S, area, tid, warp, lane);
        area ^= 1;
      } else {
        run_control<TR>(h, A, S, tid);
      }
      off += h.bytes;
    }
    consumer_sync();  // every consumer is done with this page
    if (tid == 0) mbar_arrive(empty + stage);
    if (++stage == NST) {
      stage = 0;
      phase ^= 1u;
    }
    if (quit) break;
  }
}

template <class TR>
size_t smem_for(int page_bytes, int nstages, int buf_ab, int l) {
  const size_t vec_off = ((size_t)nstages * page_bytes + 16 * (size_t)nstages + 16 + 127) & ~size_t(127);
  return vec_off + sizeof(typename TR::C) * (2 * (size_t)buf_ab + 2 * (size_t)l + 2 * (size_t)kConsumerThreads);
}

}  // namespace

size_t sweep_smem_bytes(int prec, int page_bytes, int nstages, int buf_ab, int l) {
  switch (prec) {
    case PREC_FP64: return smem_for<TF64>(page_bytes, nstages, buf_ab, l);
    case PREC_FP32: return smem_for<TF32>(page_bytes, nstages, buf_ab, l);
    default: return smem_for<TS32>(page_bytes, nstages, buf_ab, l);
  }
}

cudaError_t sweep_configure(int prec, size_t smem) {
  switch (prec) {
    case PREC_FP64:
      return cudaFuncSetAttribute(bfly_sweep_kernel<TF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case PREC_FP32:
      return cudaFuncSetAttribute(bfly_sweep_kernel<TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    default:
      return cudaFuncSetAttribute(bfly_sweep_kernel<TS32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
}

int sweep_blocks_per_sm(int prec, size_t smem) {
  int nb = 0;
  const int threads = kConsumerThreads + 32;
  cudaError_t e;
  switch (prec) {
    case PREC_FP64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bfly_sweep_kernel<TF64>, threads, smem); break;
    case PREC_FP32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bfly_sweep_kernel<TF32>, threads, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bfly_sweep_kernel<TS32>, threads, smem); break;
  }
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t sweep_launch(int prec, const SweepArgs& a, int grid, size_t smem, cudaStream_t st) {
  const dim3 block(kConsumerThreads + 32);
  switch (prec) {
    case PREC_FP64: bfly_sweep_kernel<TF64><<<grid, block, smem, st>>>(a); break;
    case PREC_FP32: bfly_sweep_kernel<TF32><<<grid, block, smem, st>>>(a); break;
    default: bfly_sweep_kernel<TS32><<<grid, block, smem, st>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace sht
