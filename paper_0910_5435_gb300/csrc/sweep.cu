// sweep.cu -- persistent butterfly sweep kernels (sm_103a).
//
// One launch applies the Legendre stage of every order m in one direction:
// synthesis (Section 2, eq. alternate_expansion, sums over k, through the
// butterfly of Section 2.2 per parity block) or analysis (the transposed
// application, Section 2.2 remark after Figure multi).
//
// Each CTA is persistent and runs a small dataflow scheduler:
//   * a producer warp pops work items (orders m) from an LPT-sorted queue
//     (atomic counter) and streams their factor pages from HBM into any free
//     stage of a ring in shared memory with 1-D TMA bulk copies
//     (cp.async.bulk, mbarrier complete_tx), recording the issue order;
//   * a parser warp follows that order, numbers the ops of every landed page
//     and publishes them in an op directory;
//   * the consumer warps each claim the next op number, wait until the op's
//     listed predecessors have completed (completion tags in shared memory),
//     and execute it alone: lanes own consecutive outputs (coalesced reads of
//     the [K][M] value block), tiny ops split the inner dimension over a few
//     lanes and reduce with warp shuffles.  There is no CTA-wide barrier; the
//     last warp to finish an op of a page returns the page to the producer.
//
// Every wait is bounded: on timeout the kernel records SHT_ERR_TIMEOUT in the
// device status word, raises the CTA abort flag, stops issuing copies, waits
// (bounded) for the copies it already issued, and returns.

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "sht_stream.h"

namespace sht {
namespace {

template <int NW>
constexpr int threads_for() { return (NW + 2) * 32; }  // consumers + producer + parser
constexpr int kMaxStages = 16;
constexpr int kDir = 1024;                            // op directory entries (ring)
constexpr int kOrd = 64;                              // page issue-order ring (>= stages)
constexpr long long kTimeoutCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr unsigned kStatusTimeout = 5;              // SHT_ERR_TIMEOUT
constexpr unsigned kStatusBadArg = 1;               // SHT_ERR_INVALID_ARG (a field's pointers)

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
// orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) writes to it
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
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
  // one accumulation chain: a full-warp DFMA holds the scheduler's FP64 pipe
  // longer than its latency, so a second chain only adds merge work
  static constexpr int kChains = 1;
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
  __device__ static Acc shfl_xor(const Acc& a, int off) {
    return {__shfl_xor_sync(0xffffffffu, a.re, off), __shfl_xor_sync(0xffffffffu, a.im, off)};
  }
  __device__ static Acc shfl_down(const Acc& a, int off) {
    return {__shfl_down_sync(0xffffffffu, a.re, off), __shfl_down_sync(0xffffffffu, a.im, off)};
  }
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
  static constexpr int kChains = 2;
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
  __device__ static Acc shfl_xor(const Acc& a, int off) {
    return {__shfl_xor_sync(0xffffffffu, a.rh, off), __shfl_xor_sync(0xffffffffu, a.rl, off),
            __shfl_xor_sync(0xffffffffu, a.ih, off), __shfl_xor_sync(0xffffffffu, a.il, off)};
  }
  __device__ static Acc shfl_down(const Acc& a, int off) {
    return {__shfl_down_sync(0xffffffffu, a.rh, off), __shfl_down_sync(0xffffffffu, a.rl, off),
            __shfl_down_sync(0xffffffffu, a.ih, off), __shfl_down_sync(0xffffffffu, a.il, off)};
  }
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

// Split float32 factors as TS32, products as float32 error-free pairs, but
// accumulated in float64: the high parts of the products in a double, their
// low parts (orders of magnitude smaller) in a float.
struct TS32A : TS32 {
  static constexpr int kChains = 1;  // float64 adds: the FP64 pipe hides the chain
  struct Acc {
    double re, im;
    float rl, il;
  };
  __device__ static Acc zero() { return {0.0, 0.0, 0.f, 0.f}; }
  __device__ static void fma1(double& s, float& sl, float2 v, float xh, float xl) {
    const float p = __fmul_rn(v.x, xh);
    float e = __fmaf_rn(v.x, xh, -p);
    e = __fmaf_rn(v.x, xl, e);
    e = __fmaf_rn(v.y, xh, e);
    s += (double)p;
    sl = __fadd_rn(sl, e);
  }
  __device__ static void fma(Acc& a, V v, const C& x) {
    fma1(a.re, a.rl, v, x.x, x.y);
    fma1(a.im, a.il, v, x.z, x.w);
  }
  __device__ static void add(Acc& a, const C& c) {
    a.re += (double)c.x;
    a.rl = __fadd_rn(a.rl, c.y);
    a.im += (double)c.z;
    a.il = __fadd_rn(a.il, c.w);
  }
  __device__ static void merge(Acc& a, const Acc& b) {
    a.re += b.re;
    a.im += b.im;
    a.rl = __fadd_rn(a.rl, b.rl);
    a.il = __fadd_rn(a.il, b.il);
  }
  __device__ static C to_c(const Acc& a) {
    const double r = a.re + (double)a.rl, i = a.im + (double)a.il;
    const float rh = __double2float_rn(r), ih = __double2float_rn(i);
    return make_float4(rh, __double2float_rn(r - (double)rh), ih, __double2float_rn(i - (double)ih));
  }
  __device__ static Acc from_c(const C& c) { return {(double)c.x + (double)c.y, (double)c.z + (double)c.w, 0.f, 0.f}; }
  __device__ static Acc shfl_xor(const Acc& a, int off) {
    return {__shfl_xor_sync(0xffffffffu, a.re, off), __shfl_xor_sync(0xffffffffu, a.im, off),
            __shfl_xor_sync(0xffffffffu, a.rl, off), __shfl_xor_sync(0xffffffffu, a.il, off)};
  }
  __device__ static Acc shfl_down(const Acc& a, int off) {
    return {__shfl_down_sync(0xffffffffu, a.re, off), __shfl_down_sync(0xffffffffu, a.im, off),
            __shfl_down_sync(0xffffffffu, a.rl, off), __shfl_down_sync(0xffffffffu, a.il, off)};
  }
};

// float32 factors and arithmetic; complex64 I/O.
struct TF32 {
  static constexpr int kChains = 2;
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
  __device__ static Acc shfl_xor(const Acc& a, int off) {
    return {__shfl_xor_sync(0xffffffffu, a.re, off), __shfl_xor_sync(0xffffffffu, a.im, off)};
  }
  __device__ static Acc shfl_down(const Acc& a, int off) {
    return {__shfl_down_sync(0xffffffffu, a.re, off), __shfl_down_sync(0xffffffffu, a.im, off)};
  }
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

// ------------------------------------------------------------ scheduler

// Shared scheduling state of one CTA.
struct Sched {
  int n_ready;    // ops published by the parser (op numbers 0 .. n_ready-1)
  int n_claimed;  // next op number to hand to a consumer warp
  int n_done;     // ops completed (any order)
  int n_issued;   // pages issued by the producer
  int quit;       // number of the QUIT op once parsed, else -1
  int abort;      // set when a bounded wait gave up
  int pending[kMaxStages];  // ops of the page in each stage not yet completed
  int order[kOrd];          // stage of the i-th issued page (i % kOrd)
  uint16_t stage_field[kMaxStages];  // field of the page in each stage (batched launches)
  uint32_t dir[kDir];       // op number % kDir -> (stage << 16) | (byte offset / 16)
  uint16_t done_tag[kDoneWindow];  // low 16 bits of the last completed op number in each slot
};

__device__ __forceinline__ int vload(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
__device__ __forceinline__ void vstore(int* p, int v) { *reinterpret_cast<volatile int*>(p) = v; }
__device__ __forceinline__ unsigned vload16(const uint16_t* p) {
  return *reinterpret_cast<const volatile uint16_t*>(p);
}

// Lane 0 polls until pred() holds (bounded), the warp then agrees on the outcome.
template <class Pred>
__device__ __forceinline__ bool warp_wait(Pred pred, Sched* S, unsigned* status, int lane) {
  int ok = 1;
  if (lane == 0) {
    if (!pred()) {
      const long long t0 = clock64();
      for (;;) {
        if (pred()) break;
        if (vload(&S->abort)) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > kTimeoutCycles) {
          atomicCAS(status, 0u, kStatusTimeout);
          vstore(&S->abort, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __threadfence_block();  // acquire what the producing warps wrote before publishing
  return ok != 0;
}

// Every lane polls its own predicate (bounded); returns when all hold.
template <class Pred>
__device__ __forceinline__ bool warp_wait_all(Pred pred, Sched* S, unsigned* status) {
  if (__all_sync(0xffffffffu, pred())) {
    __threadfence_block();
    return true;
  }
  const long long t0 = clock64();
  for (;;) {
    __nanosleep(32);
    if (__all_sync(0xffffffffu, pred())) break;
    int bad = 0;
    if ((threadIdx.x & 31) == 0) {
      if (vload(&S->abort)) bad = 1;
      else if (clock64() - t0 > kTimeoutCycles) {
        atomicCAS(status, 0u, kStatusTimeout);
        vstore(&S->abort, 1);
        bad = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, bad, 0)) return false;
  }
  __threadfence_block();  // acquire what the predecessor ops wrote
  return true;
}

// ------------------------------------------------------------ ops

template <class TR>
struct Vecs {
  using C = typename TR::C;
  C* base;
  int buf_ab;
  __device__ C* buf(int id) const { return base + (size_t)id * buf_ab; }
};

__device__ __forceinline__ size_t tri_off(int m, int L) { return (size_t)m * L - (size_t)m * (m - 1) / 2; }

template <bool GLOBAL, class T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (GLOBAL) {
    return __ldcs(p);  // streamed once per launch: evict-first
  } else {
    return *p;
  }
}

// Accumulates lane o's dot product over the inner indices s = q, q + ks, ...
// Values come from shared memory (pages) or straight from global memory; the
// global variant keeps 8 rows of loads in flight per lane (the latency of a
// streamed HBM read is hidden by the loads of the same warp, not only by
// other warps).
template <class TR, bool GLOBAL>
__device__ __forceinline__ typename TR::Acc gemv_dot(const typename TR::V* val, const typename TR::C* in,
                                                     const uint16_t* idx, bool gather, int M, int K, int o, int q,
                                                     int ks) {
  using C = typename TR::C;
  using V = typename TR::V;
  using Acc = typename TR::Acc;
  constexpr int U = GLOBAL ? 8 : 4;
  // TR::kChains accumulation chains per lane; each extra chain costs a merge
  constexpr int NC = TR::kChains;
  Acc a[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) a[c] = TR::zero();
  int s = q;
  for (; s + (U - 1) * ks < K; s += U * ks) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ldv<GLOBAL>(val + (size_t)(s + u * ks) * M + o);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int su = s + u * ks;
      TR::fma(a[u % NC], v[u], in[gather ? (int)idx[su] : su]);
    }
  }
  for (; s < K; s += ks) TR::fma(a[0], ldv<GLOBAL>(val + (size_t)s * M + o), in[gather ? (int)idx[s] : s]);
#pragma unroll
  for (int c = 1; c < NC; ++c) TR::merge(a[0], a[c]);
  return a[0];
}

// floor(32 / M) for M = 0..32, and ceil(65536 / d) for d = 0..32.
__constant__ unsigned char c_lanes_per_out[33] = {0, 32, 16, 10, 8, 6, 5, 4, 4, 3, 3, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
__constant__ unsigned c_inv16[33] = {0, 65536, 32768, 21846, 16384, 13108, 10923, 9363, 8192, 7282, 6554, 5958, 5462, 5042, 4682, 4370, 4096, 3856, 3641, 3450, 3277, 3121, 2979, 2850, 2731, 2622, 2521, 2428, 2341, 2260, 2185, 2115, 2048};

// What an op needs of its field: the launch's own arguments, or one field
// of a batched launch.
struct FieldCtx {
  const uint8_t* values;
  const void* in;
  void* out;
  const double* prescale;
  const double2* twiddle;
  int l;
};
__device__ __forceinline__ FieldCtx field_ctx(const SweepArgs& A, int f) {
  if (!A.fields) return {A.values, A.in, A.out, A.prescale, A.twiddle, A.l};
  const FieldDesc& d = A.fields[f];
  return {d.values, A.field_in[f], A.field_out[f], d.prescale, d.twiddle, d.l};
}

// One compute op (SYN_INTERP, DENSE, DENSE_G, ANA_INTERP), executed by one warp.
template <class TR>
__device__ __forceinline__ void run_gemv(const OpHdr& h, const uint8_t* op, const Vecs<TR>& S, const FieldCtx& A,
                                         int lane, const uint8_t* staged) {
  using C = typename TR::C;
  using V = typename TR::V;
  using Acc = typename TR::Acc;
  using IO = typename TR::IO;
  const int M = h.M, K = h.K;
  const uint16_t* idx = reinterpret_cast<const uint16_t*>(op + sizeof(OpHdr)) + h.npred;
  // values: staged in this warp's slot, else streamed from the value region,
  // else inside the page after the index area
  const bool from_global = staged == nullptr && (h.flags & F_VALUES_APART) != 0;
  const V* val = staged ? reinterpret_cast<const V*>(staged)
                        : from_global ? reinterpret_cast<const V*>(A.values + (size_t)h.vref * 16)
                                      : reinterpret_cast<const V*>(op + sizeof(OpHdr) + (size_t)h.idx16 * 16);
  const C* in = S.buf(h.in_buf) + h.io;
  C* out = S.buf(h.out_buf) + h.oo;
  const bool gather = (h.kind == OP_SYN_INTERP);
  const bool accum = (h.flags & F_ACCUM) != 0;
  if (M > 0) {
    // ks = floor(32 / M) lanes per output (not only powers of two, so that
    // up to 32 - ks + 1 lanes work); lane = o * ks + q.  Both divisions come
    // from a table: lane / ks = (lane * ceil(2^16 / ks)) >> 16 holds exactly
    // for lane < 32 and ks <= 32.
    const int ks = c_lanes_per_out[M];
    const int o = (lane * c_inv16[ks]) >> 16, q = lane - o * ks;
    Acc a0 = TR::zero();
    if (o < M)
      a0 = from_global ? gemv_dot<TR, true>(val, in, idx, gather, M, K, o, q, ks)
                       : gemv_dot<TR, false>(val, in, idx, gather, M, K, o, q, ks);
    // segmented tree: after the step with offset d, lane q holds the sum over
    // q .. min(q + 2d - 1, ks - 1) of its segment
    for (int off = 1; off < ks; off <<= 1) {
      const Acc b = TR::shfl_down(a0, off);
      if (q + off < ks) TR::merge(a0, b);
    }
    if (q == 0 && o < M) {
      switch (h.kind) {
        case OP_SYN_INTERP:
          TR::add(a0, in[idx[K + o]]);
          out[o] = TR::to_c(a0);
          break;
        case OP_DENSE:
          out[o] = TR::to_c(a0);
          break;
        case OP_ANA_INTERP: {
          const int pos = idx[o];
          if (accum) TR::add(a0, out[pos]);
          out[pos] = TR::to_c(a0);
          break;
        }
        case OP_DENSE_G: {
          const int l = A.l;
          const int i = h.oo + o;
          IO v = TR::to_io(TR::to_c(a0));
          if (A.twiddle) v = TR::io_cmul(v, A.twiddle[h.a1]);
          IO* G = reinterpret_cast<IO*>(A.out) + (size_t)h.a1 * (2 * l);
          if (accum) {
            G[l + i] = TR::io_add(G[l + i], v);
            G[l - 1 - i] = TR::io_sub(G[l - 1 - i], v);
          } else {
            G[l + i] = v;
            G[l - 1 - i] = v;
          }
          break;
        }
        default:
          break;
      }
    }
  }
  if (h.kind == OP_ANA_INTERP && (h.flags & F_SKEL)) {
    const uint16_t* skel = idx + M;
    for (int t = lane; t < h.nskel; t += 32) {
      const int pos = skel[t];
      if (accum) {
        Acc r = TR::from_c(out[pos]);
        TR::add(r, in[t]);
        out[pos] = TR::to_c(r);
      } else {
        out[pos] = in[t];
      }
    }
  }
}

// One control op over the element range [oo, oo + M), executed by one warp.
template <class TR>
__device__ __forceinline__ void run_control(const OpHdr& h, const Vecs<TR>& S, const FieldCtx& A, int lane) {
  using C = typename TR::C;
  using IO = typename TR::IO;
  const int l = A.l, L = 2 * l;
  const int m = (int)h.a1;
  const int n = h.M;
  const int parity = h.a0 & 1, base = h.a0 >> 1;  // GATHER / SCATTER / FOLD
  switch (h.kind) {
    case OP_GATHER: {
      const IO* beta = reinterpret_cast<const IO*>(A.in) + tri_off(m, L) + parity;
      C* dst = S.buf(h.out_buf) + base;
      for (int j = h.oo + lane; j < h.oo + n; j += 32) dst[j] = TR::from_io(beta[2 * (size_t)j]);
      break;
    }
    case OP_SCATTER: {
      IO* beta = reinterpret_cast<IO*>(A.out) + tri_off(m, L) + parity;
      const C* src = S.buf(h.in_buf) + base;
      for (int j = h.io + lane; j < h.io + n; j += 32) beta[2 * (size_t)j] = TR::to_io(src[j]);
      break;
    }
    case OP_FOLD: {
      const IO* G = reinterpret_cast<const IO*>(A.in) + (size_t)m * L;
      C* dst = S.buf(h.out_buf) + base;
      for (int r = h.oo + lane; r < h.oo + n; r += 32) {
        IO gp = G[l + r], gm = G[l - 1 - r];
        if (A.twiddle) {
          gp = TR::io_cmul(gp, A.twiddle[m]);
          gm = TR::io_cmul(gm, A.twiddle[m]);
        }
        IO e = parity ? TR::io_sub(gp, gm) : TR::io_add(gp, gm);
        if (A.prescale) e = TR::io_scale(e, A.prescale[r]);
        dst[r] = TR::from_io(e);
      }
      break;
    }
    case OP_CLEAR: {
      C* dst = S.buf(h.out_buf);
      for (int j = h.oo + lane; j < h.oo + n; j += 32) dst[j] = TR::czero();
      break;
    }
    case OP_GZERO: {
      IO* G = reinterpret_cast<IO*>(A.out) + (size_t)m * L;
      for (int r = h.oo + lane; r < h.oo + n; r += 32) {
        G[l + r] = TR::io_zero();
        G[l - 1 - r] = TR::io_zero();
      }
      break;
    }
    default:
      break;
  }
}

// ------------------------------------------------------------ roles

__device__ __forceinline__ void trace_add(const SweepArgs& A, int slot, unsigned long long v) {
  if (A.trace && v) atomicAdd(A.trace + slot, v);
}

__device__ void producer_loop(const SweepArgs& A, uint8_t* stages, uint64_t* full, uint64_t* empty, Sched* S) {
  const uint32_t PB = (uint32_t)A.page_bytes;
  const int NST = A.nstages;
  volatile int* abort_flag = &S->abort;
  int uses[kMaxStages];  // pages copied into each stage so far
  for (int s = 0; s < kMaxStages; ++s) uses[s] = 0;
  int issued = 0;
  unsigned long long c_wait = 0;
  // any stage whose previous page has been fully consumed may be refilled
  auto free_stage = [&]() -> int {
    const long long t0 = clock64();
    for (int spin = 0;; ++spin) {
      for (int s = 0; s < NST; ++s)
        if (mbar_try_wait(empty + s, (uint32_t)((uses[s] & 1) ^ 1))) {
          c_wait += clock64() - t0;
          return s;
        }
      if (*abort_flag) return -1;
      if (clock64() - t0 > kTimeoutCycles) {
        atomicCAS(A.status, 0u, kStatusTimeout);
        *abort_flag = 1;
        return -1;
      }
      __nanosleep(64);
    }
  };
  auto issue = [&](int s, const uint8_t* pages, uint64_t page, int field) {
    S->stage_field[s] = (uint16_t)field;  // read by the op's warps while the page is pending
    fence_proxy_async();
    mbar_arrive_expect_tx(full + s, PB);
    bulk_g2s(stages + (size_t)s * PB, pages + (size_t)page * PB, PB, full + s);
    ++uses[s];
    S->order[issued % kOrd] = s;
    ++issued;
    __threadfence_block();
    vstore(&S->n_issued, issued);
  };
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
    const int field = A.fields ? (int)e.m : 0;
    const uint8_t* pages = A.fields ? A.fields[field].pages : A.pages;
    if (A.fields) {
      // a batched field's input and output come from device arrays: check
      // them before any page of the field is issued
      const uintptr_t io = reinterpret_cast<uintptr_t>(A.field_in[field]) |
                           reinterpret_cast<uintptr_t>(A.field_out[field]);
      if (!A.field_in[field] || !A.field_out[field] || (io & (uintptr_t)(A.io_align - 1))) {
        atomicCAS(A.status, 0u, kStatusBadArg);
        *abort_flag = 1;
        ok = false;
        break;
      }
    }
    for (uint32_t pg = 0; pg < e.n_pages; ++pg) {
      const int s = free_stage();
      if (s < 0) {
        ok = false;
        break;
      }
      issue(s, pages, e.first_page + pg, field);
    }
    if (!ok) break;
  }
  if (ok) {
    const int s = free_stage();
    if (s >= 0) issue(s, A.pages, A.quit_page, 0);
  }
  // never leave the CTA with bulk copies still landing in its shared memory
  for (int s = 0; s < NST; ++s)
    if (uses[s] > 0) wait_bounded(full + s, (uint32_t)((uses[s] - 1) & 1), A.status, abort_flag);
  trace_add(A, TR_PROD_WAIT, c_wait);
}

// One warp publishes the ops of each landed page, in issue order, from the
// page's op table: lanes write up to 32 directory entries at once.
__device__ void parser_loop(const SweepArgs& A, const uint8_t* stages, uint64_t* full, uint64_t* empty,
                            Sched* S, int lane) {
  const size_t PB = (size_t)A.page_bytes;
  uint32_t parsed_bits = 0;  // bit s: parity of the next completion of stage s
  int ticket = 0;
  unsigned long long c_wait = 0;
  for (int k = 0;; ++k) {
    const long long w0 = clock64();
    // the k-th issued page: which stage, then wait for its bytes
    int stage = 0, ok = 1;
    if (lane == 0) {
      while (vload(&S->n_issued) <= k) {
        if (vload(&S->abort) || clock64() - w0 > kTimeoutCycles) {
          if (!vload(&S->abort)) {
            atomicCAS(A.status, 0u, kStatusTimeout);
            vstore(&S->abort, 1);
          }
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
      if (ok) {
        __threadfence_block();
        stage = vload(&S->order[k % kOrd]);
        ok = wait_bounded(full + stage, (parsed_bits >> stage) & 1u, A.status, &S->abort) ? 1 : 0;
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return;
    stage = __shfl_sync(0xffffffffu, stage, 0);
    mbar_try_wait(full + stage, (parsed_bits >> stage) & 1u);  // each lane's acquire of the page bytes
    parsed_bits ^= 1u << stage;
    c_wait += clock64() - w0;
    const uint8_t* page = stages + (size_t)stage * PB;
    const int n = *reinterpret_cast<const uint16_t*>(page + PB - 2);
    if (n == kQuitPage) {
      if (lane == 0) {
        __threadfence_block();
        vstore(&S->quit, ticket);
        trace_add(A, TR_PARSE_WAIT, c_wait);
      }
      return;
    }
    if (lane == 0) {
      vstore(&S->pending[stage], n);
      if (n == 0) mbar_arrive(empty + stage);  // nothing to execute: the stage is free again
    }
    __syncwarp();
    for (int i0 = 0; i0 < n; i0 += 32) {
      const int cnt = min(32, n - i0);
      // entry u reuses the slot of op u - kDir: that op must have completed
      // (so its entry was read); its completion tag says so
      const int u = ticket + lane;
      const int prev = (lane < cnt) ? u - kDir : -1;
      const uint16_t* tag = S->done_tag + (prev >= 0 ? prev % kDoneWindow : 0);
      const unsigned want = (unsigned)(prev & 0xffff);
      if (!warp_wait_all([&] { return prev < 0 || vload16(tag) == want; }, S, A.status)) return;
      if (lane < cnt) {
        const uint32_t off16 = *reinterpret_cast<const uint16_t*>(page + PB - 4 - 2 * (size_t)(i0 + lane));
        S->dir[(ticket + lane) % kDir] = ((uint32_t)stage << 16) | off16;
      }
      __syncwarp();
      ticket += cnt;
      if (lane == 0) {
        __threadfence_block();
        vstore(&S->n_ready, ticket);
      }
    }
  }
}

// An op claimed by a consumer warp.
struct Claim {
  int t;               // op number
  int stage;           // ring stage of its page
  const uint8_t* op;   // header in the page
  OpHdr h;
  int slot;            // staging slot of its values (0 / 1), or -1
  int field;           // field of its page (batched launches)
  uint32_t vbytes;     // bytes of its value block
  bool deferred;       // its copy waits for the warp's only slot to be read
};

template <class TR>
__device__ void consumer_loop(const SweepArgs& A, const uint8_t* stages, uint64_t* empty, Sched* S,
                              const Vecs<TR>& V, int lane, uint8_t* my_slots, uint64_t* my_bars) {
  using Val = typename TR::V;
  const int kSlotBytes = A.slot_bytes;
  const size_t PB = (size_t)A.page_bytes;
  unsigned long long c_exec = 0, c_ready = 0, c_dep = 0, c_val = 0, n_ops = 0;
  unsigned long long c_gemv = 0, c_ctl = 0, c_done = 0, n_gemv = 0, n_ctl = 0;
  const bool tracing = A.trace != nullptr;  // cycle counts only while tracing
  uint32_t slot_phase = 0u;  // bit s: parity of slot s's next completion
  uint32_t inflight = 0u;    // bit s: a copy into slot s has not been waited for
  int next_slot = 0;
  // with one slot per warp the next op's copy starts only once the current
  // op has read the slot (other warps cover the copy); with two it travels
  // while the current op runs
  const bool one_slot = A.warp_slots == 1;

  // Op numbers are claimed in order; an op is "opened" once it is published:
  // its header is read and (values kept apart) the bulk copy of its value
  // block into a free slot starts.  A warp that holds an unexecuted op only
  // polls for the next one (that op's page may be waiting for the held op's
  // page to drain); it blocks on publication only when it holds nothing.
  auto claim_number = [&]() -> int {
    int t = 0;
    if (lane == 0) t = atomicAdd(&S->n_claimed, 1);
    return __shfl_sync(0xffffffffu, t, 0);
  };
  auto start_copy = [&](Claim& c) {
    if (lane == 0) {
      fence_proxy_async();  // earlier reads of this slot precede the copy into it
      mbar_arrive_expect_tx(my_bars + c.slot, c.vbytes);
      const uint8_t* vals = A.fields ? A.fields[c.field].values : A.values;
      bulk_g2s(my_slots + (size_t)c.slot * kSlotBytes, vals + (size_t)c.h.vref * 16, c.vbytes, my_bars + c.slot);
    }
    inflight |= 1u << c.slot;
    c.deferred = false;
  };
  // 1: opened, 0: t is past the end of the stream, 2: not yet published
  // (poll only), -1: aborted.  holding: the warp holds an op not yet run.
  auto open = [&](int t, Claim& c, bool block, bool holding) -> int {
    auto published = [&] {
      const int q = vload(&S->quit);
      return vload(&S->n_ready) > t || (q >= 0 && t >= q);
    };
    if (block) {
      const long long t0 = clock64();
      if (!warp_wait(published, S, A.status, lane)) return -1;
      c_ready += clock64() - t0;
    } else {
      int ok = 0;
      if (lane == 0) ok = published() ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, ok, 0)) return 2;
      __threadfence_block();
    }
    const int q = vload(&S->quit);
    if (q >= 0 && t >= q) return 0;
    const uint32_t e = S->dir[t % kDir];
    __syncwarp();
    c.t = t;
    c.stage = (int)(e >> 16);
    c.op = stages + (size_t)c.stage * PB + ((size_t)(e & 0xffffu) << 4);
    c.h = *reinterpret_cast<const OpHdr*>(c.op);
    c.field = A.fields ? (int)S->stage_field[c.stage] : 0;
    c.slot = -1;
    c.deferred = false;
    c.vbytes = (uint32_t)((sizeof(Val) * c.h.M * c.h.K + 15) & ~size_t(15));
    // a block larger than a slot (not emitted by the planner) is streamed instead
    if ((c.h.flags & F_VALUES_APART) && my_slots && c.vbytes <= (uint32_t)kSlotBytes) {
      c.slot = one_slot ? 0 : next_slot;
      next_slot ^= 1;
      if (one_slot && holding)
        c.deferred = true;
      else
        start_copy(c);
    }
    return 1;
  };

  Claim cur, nxt;
  int rc = open(claim_number(), cur, true, false);
  while (rc == 1) {
    const int tn = claim_number();
    int rn = open(tn, nxt, false, cur.slot >= 0);  // the next op's values travel while this one runs
    if (rn < 0) break;
    const long long t1 = tracing ? clock64() : 0;
    bool ok;
    if (cur.h.kind == OP_JOIN && (cur.h.flags & F_ITEM_START)) {
      // a work item starts once every earlier op of this CTA has completed
      ok = warp_wait([&] { return vload(&S->n_done) >= cur.t; }, S, A.status, lane);
    } else {
      // lanes watch the listed predecessors (32 at a time)
      const uint16_t* pred = reinterpret_cast<const uint16_t*>(cur.op + sizeof(OpHdr));
      ok = true;
      for (int base = 0; base < cur.h.npred && ok; base += 32) {
        const int i = base + lane;
        const int u = (i < cur.h.npred) ? cur.t - (int)pred[i] : -1;
        const unsigned want = (unsigned)(u & 0xffff);
        const uint16_t* slot = S->done_tag + (u >= 0 ? (u % kDoneWindow) : 0);
        ok = warp_wait_all([&] { return u < 0 || vload16(slot) == want; }, S, A.status);
      }
    }
    if (!ok) break;
    const long long t2 = tracing ? clock64() : 0;
    const uint8_t* staged = nullptr;
    if (cur.slot >= 0) {
      uint64_t* bar = my_bars + cur.slot;
      const uint32_t ph = (slot_phase >> cur.slot) & 1u;
      if (!warp_wait([&] { return mbar_try_wait(bar, ph); }, S, A.status, lane)) break;
      mbar_try_wait(bar, ph);  // each lane's own acquire of the copied bytes
      slot_phase ^= 1u << cur.slot;
      inflight &= ~(1u << cur.slot);
      staged = my_slots + (size_t)cur.slot * kSlotBytes;
    }
    const long long t3 = tracing ? clock64() : 0;
    const bool is_gemv = cur.h.kind >= OP_SYN_INTERP && cur.h.kind <= OP_ANA_INTERP;
    if (is_gemv)
      run_gemv<TR>(cur.h, cur.op, V, field_ctx(A, cur.field), lane, staged);
    else if (cur.h.kind != OP_JOIN)
      run_control<TR>(cur.h, V, field_ctx(A, cur.field), lane);
    const long long t3b = tracing ? clock64() : 0;
    if (tracing) {
      if (is_gemv) {
        c_gemv += t3b - t3;
        ++n_gemv;
      } else {
        c_ctl += t3b - t3;
        ++n_ctl;
      }
    }
    __threadfence_block();  // this op's results are visible before it is marked done
    __syncwarp();
    if (lane == 0) {
      *reinterpret_cast<volatile uint16_t*>(&S->done_tag[cur.t % kDoneWindow]) = (uint16_t)(cur.t & 0xffff);
      atomicAdd(&S->n_done, 1);
      if (atomicSub(&S->pending[cur.stage], 1) == 1) mbar_arrive(empty + cur.stage);
    }
    const long long t4 = tracing ? clock64() : 0;
    if (tracing) {
      c_done += t4 - t3b;
      c_dep += t2 - t1;
      c_val += t3 - t2;
      c_exec += t4 - t3;
      ++n_ops;
    }
    if (rn == 1 && nxt.deferred) start_copy(nxt);  // the slot has been read
    if (rn == 2) rn = open(tn, nxt, true, false);  // holds nothing now
    if (rn != 1) break;
    cur = nxt;
  }
  // never leave with a bulk copy still landing in this warp's slots
  for (int s = 0; s < 2; ++s)
    if (((inflight >> s) & 1u) && lane == 0) wait_bounded(my_bars + s, (slot_phase >> s) & 1u, A.status, &S->abort);
  __syncwarp();
  if (lane == 0) {
    trace_add(A, TR_EXEC, c_exec);
    trace_add(A, TR_WAIT_READY, c_ready);
    trace_add(A, TR_WAIT_DEP, c_dep);
    trace_add(A, TR_WAIT_VALUES, c_val);
    trace_add(A, TR_OPS, n_ops);
    trace_add(A, TR_EXEC_GEMV, c_gemv);
    trace_add(A, TR_EXEC_CTL, c_ctl);
    trace_add(A, TR_COMPLETE, c_done);
    trace_add(A, TR_N_GEMV, n_gemv);
    trace_add(A, TR_N_CTL, n_ctl);
  }
}

// Shared-memory layout of a sweep CTA, used by the kernel and by the host
// sizing alike: [pages: nst x pb][full, empty barriers: 2 x nst][slot
// barriers: 2 x nw][Sched] | 128-aligned vectors | 128-aligned staging
// slots (nw x warp_slots x slot_bytes).
__host__ __device__ inline size_t sweep_vec_offset(int nst, size_t pb, int nw) {
  return ((size_t)nst * pb + 16 * (size_t)nst + 16 * (size_t)nw + sizeof(Sched) + 127) & ~size_t(127);
}
__host__ __device__ inline size_t sweep_slot_offset(size_t vec_off, size_t vec_bytes) {
  return (vec_off + vec_bytes + 127) & ~size_t(127);
}

template <class TR, int NW>
__global__ void __launch_bounds__(threads_for<NW>()) bfly_sweep_kernel(const SweepArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NST = A.nstages;
  const size_t PB = (size_t)A.page_bytes;
  uint8_t* stages = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * PB);
  uint64_t* empty = full + NST;
  uint64_t* slot_bars = empty + NST;  // 2 per consumer warp
  Sched* S = reinterpret_cast<Sched*>(slot_bars + 2 * NW);
  const size_t vec_off = sweep_vec_offset(NST, PB, NW);
  const Vecs<TR> V{reinterpret_cast<typename TR::C*>(smem + vec_off), A.buf_ab};
  uint8_t* slots =
      A.staged ? smem + sweep_slot_offset(vec_off, sizeof(typename TR::C) * (size_t)A.num_vecs * A.buf_ab) : nullptr;

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int s = 0; s < 2 * NW; ++s) mbar_init(slot_bars + s, 1);
    S->n_ready = 0;
    S->n_claimed = 0;
    S->n_done = 0;
    S->n_issued = 0;
    S->quit = -1;
    S->abort = 0;
    fence_mbar_init();
  }
  // completion tags start as "op slot - window", which no op number in the
  // first window matches
  for (int i = tid; i < kDoneWindow; i += blockDim.x) S->done_tag[i] = (uint16_t)((i - kDoneWindow) & 0xffff);
  __syncthreads();

  if (warp == NW) {
    if (lane == 0) producer_loop(A, stages, full, empty, S);
  } else if (warp == NW + 1) {
    parser_loop(A, stages, full, empty, S, lane);
  } else {
    const int ws = A.warp_slots == 1 ? 1 : 2;
    consumer_loop<TR>(A, stages, empty, S, V, lane, slots ? slots + (size_t)warp * ws * A.slot_bytes : nullptr,
                      slot_bars + 2 * warp);
  }
}

template <class TR>
size_t smem_for(int page_bytes, int nstages, int buf_ab, int num_vecs, int nw, int slot_bytes, int warp_slots) {
  const size_t vec_off = sweep_vec_offset(nstages, (size_t)page_bytes, nw);
  const size_t vec_bytes = sizeof(typename TR::C) * (size_t)num_vecs * (size_t)buf_ab;
  if (slot_bytes <= 0) return vec_off + vec_bytes;
  return sweep_slot_offset(vec_off, vec_bytes) + (size_t)nw * (warp_slots == 1 ? 1 : 2) * slot_bytes;
}

}  // namespace

size_t sweep_smem_bytes(int prec, int page_bytes, int nstages, int buf_ab, int num_vecs, int nw, int slot_bytes,
                        int warp_slots) {
  switch (prec) {
    case PREC_FP64: return smem_for<TF64>(page_bytes, nstages, buf_ab, num_vecs, nw, slot_bytes, warp_slots);
    case PREC_FP32: return smem_for<TF32>(page_bytes, nstages, buf_ab, num_vecs, nw, slot_bytes, warp_slots);
    case PREC_SPLIT32_ACC64: return smem_for<TS32A>(page_bytes, nstages, buf_ab, num_vecs, nw, slot_bytes, warp_slots);
    default: return smem_for<TS32>(page_bytes, nstages, buf_ab, num_vecs, nw, slot_bytes, warp_slots);
  }
}

namespace {

// Host dispatch over (precision, consumer warps).
template <class TR>
const void* kernel_ptr(int nw) {
  switch (nw) {
    case 8: return reinterpret_cast<const void*>(bfly_sweep_kernel<TR, 8>);
    case 12: return reinterpret_cast<const void*>(bfly_sweep_kernel<TR, 12>);
    default: return reinterpret_cast<const void*>(bfly_sweep_kernel<TR, 16>);
  }
}
const void* kernel_for(int prec, int nw) {
  switch (prec) {
    case PREC_FP64: return kernel_ptr<TF64>(nw);
    case PREC_FP32: return kernel_ptr<TF32>(nw);
    case PREC_SPLIT32_ACC64: return kernel_ptr<TS32A>(nw);
    default: return kernel_ptr<TS32>(nw);
  }
}

}  // namespace

cudaError_t sweep_configure(int prec, size_t smem) {
  for (int nw : {8, 12, 16}) {
    cudaError_t e = cudaFuncSetAttribute(kernel_for(prec, nw), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int sweep_blocks_per_sm(int prec, int nw, size_t smem) {
  int nb = 0;
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_for(prec, nw), (nw + 2) * 32, smem);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

bool sweep_choose(int prec, int page_bytes, int buf_ab, int num_vecs, int nw, int slot_bytes, int nstages,
                  size_t optin, SweepConfig* c, int warp_slots) {
  c->nw = nw;
  c->warp_slots = warp_slots == 1 ? 1 : 2;
  // staged values need their slots next to a ring of at least two pages
  c->staged = slot_bytes > 0 &&
              sweep_smem_bytes(prec, page_bytes, 2, buf_ab, num_vecs, nw, slot_bytes, c->warp_slots) <= optin;
  c->slot_bytes = c->staged ? slot_bytes : 0;
  c->nstages = 0;
  c->ctas_per_sm = 0;
  c->smem = 0;
  for (int nst = (nstages > 0 ? nstages : 8); nst >= (nstages > 0 ? nstages : 2); --nst) {
    const size_t sm = sweep_smem_bytes(prec, page_bytes, nst, buf_ab, num_vecs, nw, c->slot_bytes, c->warp_slots);
    if (sm > optin) continue;
    const int ctas = std::min(2, sweep_blocks_per_sm(prec, nw, sm));
    const bool better = (ctas > c->ctas_per_sm && (nst >= 3 || c->ctas_per_sm == 0)) || c->ctas_per_sm == 0;
    if (better) {
      c->nstages = nst;
      c->ctas_per_sm = ctas;
      c->smem = sm;
    }
  }
  return c->nstages > 0;
}

cudaError_t sweep_launch(int prec, int nw, const SweepArgs& a, int grid, size_t smem, cudaStream_t st) {
  if (a.nstages < 1 || a.nstages > kMaxStages) return cudaErrorInvalidValue;
  if (nw != 8 && nw != 12 && nw != 16) return cudaErrorInvalidValue;
  void* args[] = {const_cast<SweepArgs*>(&a)};
  return cudaLaunchKernel(kernel_for(prec, nw), dim3(grid), dim3((nw + 2) * 32), args, smem, st);
}

}  // namespace sht
