// sweep.cu -- persistent butterfly sweep kernels (sm_103a).
//
// One launch applies the Legendre stage of every order m in one direction:
// synthesis (Section 2, eq. alternate_expansion, sums over k, through the
// butterfly of Section 2.2 per parity block) or analysis (the transposed
// application, Section 2.2 remark after Figure multi).
//
// Each CTA is persistent and takes work items (orders m) from an LPT-sorted
// queue (an atomic counter).  The planner has already scheduled every op of
// an item onto one of the CTA's warps, so a warp only walks its own list:
//   * its records (op header, the warps it waits for, index lists) arrive in
//     1-D bulk copies (cp.async.bulk, mbarrier complete_tx) into a two-chunk
//     ring of its own, a chunk ahead of the one it reads;
//   * the values of its next op are bulk-copied into its staging slot as soon
//     as the current op has read the slot, so the copy overlaps the current
//     op's end and the next op's waits;
//   * before an op it waits until the listed warps have published enough
//     completed ops (one progress word per warp in shared memory), then
//     executes the op alone: lanes own consecutive outputs (coalesced reads
//     of the [K][M] value block), ops with fewer outputs split the inner
//     dimension over a few lanes and reduce with warp shuffles (in float64
//     with the real and imaginary sums split between lane pairs, and float64
//     ops whose outputs would leave lanes idle cut into 32 equal chunks of
//     products instead); then it publishes its progress if another warp
//     waits for it;
//   * all warps meet at the end of an item (the next item reuses the shared
//     vectors); warp 0 fetches the next item's number during the current one.
// There is no producer, parser, op directory, claim or completion tag: the
// per-op protocol is a few shared-memory words.  A single-block launch (the
// Gauss-Jacobi form) runs one stage of a level-by-level schedule instead,
// with plain vector I/O and the vectors in global memory (SweepArgs).
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
  // the reduction tree splits the components between lane pairs (run_gemv)
  static constexpr bool kSplitComponents = true;
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
  __device__ static Acc shfl_idx(const Acc& a, int src) {
    return {__shfl_sync(0xffffffffu, a.re, src), __shfl_sync(0xffffffffu, a.im, src)};
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
  static constexpr bool kSplitComponents = false;
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
  static constexpr bool kSplitComponents = false;
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

// ------------------------------------------------------------ ops

// The shared vectors of one item: for each field f of its group, vectors
// A and B of buf_ab elements (field-major: [f][A, B][buf_ab]).
template <class TR>
struct Vecs {
  using C = typename TR::C;
  C* base;
  int buf_ab;
  __device__ C* buf(int id, int f = 0) const { return base + ((size_t)f * kNumVecs + id) * buf_ab; }
};

__device__ __forceinline__ size_t tri_off(int m, int L) { return (size_t)m * L - (size_t)m * (m - 1) / 2; }

// Accumulates lane o's dot product over the inner indices s = q, q + ks, ...
// of the value block staged in shared memory.
template <class TR>
__device__ __forceinline__ typename TR::Acc gemv_dot(const typename TR::V* val, const typename TR::C* in,
                                                     const uint16_t* idx, bool gather, int M, int K, int o, int q,
                                                     int ks) {
  using V = typename TR::V;
  using Acc = typename TR::Acc;
  constexpr int U = 4;
  // TR::kChains accumulation chains per lane; each extra chain costs a merge
  constexpr int NC = TR::kChains;
  Acc a[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) a[c] = TR::zero();
  int s = q;
  for (; s + (U - 1) * ks < K; s += U * ks) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = val[(size_t)(s + u * ks) * M + o];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int su = s + u * ks;
      TR::fma(a[u % NC], v[u], in[gather ? (int)idx[su] : su]);
    }
  }
  for (; s < K; s += ks) TR::fma(a[0], val[(size_t)s * M + o], in[gather ? (int)idx[s] : s]);
#pragma unroll
  for (int c = 1; c < NC; ++c) TR::merge(a[0], a[c]);
  return a[0];
}

// The same for the fields 0..nf-1 of a group (nf <= FG): each staged value
// is loaded once and applied to every field's input, in the same order and
// with the same chains per field as gemv_dot (the results are the same bits).
template <class TR, int FG>
__device__ __forceinline__ void gemv_dot_fields(const typename TR::V* val, const typename TR::C* const* in,
                                                const uint16_t* idx, bool gather, int M, int K, int o, int q,
                                                int ks, int nf, typename TR::Acc (&out)[FG]) {
  using V = typename TR::V;
  using Acc = typename TR::Acc;
  constexpr int U = 4;
  constexpr int NC = TR::kChains;
  Acc a[FG][NC];
#pragma unroll
  for (int f = 0; f < FG; ++f)
#pragma unroll
    for (int c = 0; c < NC; ++c) a[f][c] = TR::zero();
  int s = q;
  for (; s + (U - 1) * ks < K; s += U * ks) {
    V v[U];
    int xi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int su = s + u * ks;
      v[u] = val[(size_t)su * M + o];
      xi[u] = gather ? (int)idx[su] : su;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int f = 0; f < FG; ++f)
        if (f < nf) TR::fma(a[f][u % NC], v[u], in[f][xi[u]]);
  }
  for (; s < K; s += ks) {
    const V v = val[(size_t)s * M + o];
    const int xi = gather ? (int)idx[s] : s;
#pragma unroll
    for (int f = 0; f < FG; ++f)
      if (f < nf) TR::fma(a[f][0], v, in[f][xi]);
  }
#pragma unroll
  for (int f = 0; f < FG; ++f) {
#pragma unroll
    for (int c = 1; c < NC; ++c) TR::merge(a[f][0], a[f][c]);
    out[f] = a[f][0];
  }
}

// Flattened lane mapping (float64 ops whose outputs do not fill the lanes):
// the op's M x K products, taken output by output (w = o K + s), are cut into
// 32 contiguous chunks of c = ceil(M K / 32), one per lane.  As c <= K, a
// chunk meets at most two outputs: the lane sums the part of its first output
// in head and the part of the next one in tail (zero if the chunk does not
// reach it).  Every lane then runs c products, against ceil(K / floor(32 / M))
// with one or more lanes per output; the outputs' sums are put together in
// flat_combine.
template <class TR, int FG>
__device__ __forceinline__ void flat_dot(const typename TR::V* val, const typename TR::C* const* in,
                                         const uint16_t* idx, bool gather, int M, int K, int lane, int nf,
                                         typename TR::Acc (&head)[FG], typename TR::Acc (&tail)[FG]) {
  using V = typename TR::V;
  const int W = M * K, c = (W + 31) >> 5;
  const int w0 = min(lane * c, W), w1 = min(w0 + c, W);
  int o = w0 / K, s = w0 - o * K;
  bool crossed = false;
#pragma unroll
  for (int f = 0; f < FG; ++f) tail[f] = TR::zero();
  for (int w = w0; w < w1; ++w) {
    const V v = val[s * M + o];
    const int xi = gather ? (int)idx[s] : s;
#pragma unroll
    for (int f = 0; f < FG; ++f)
      if (f < nf) TR::fma(tail[f], v, in[f][xi]);
    if (++s == K) {  // the chunk passes into the next output
      s = 0;
      ++o;
      if (!crossed) {
#pragma unroll
        for (int f = 0; f < FG; ++f) {
          head[f] = tail[f];
          tail[f] = TR::zero();
        }
        crossed = true;
      }
    }
  }
  if (!crossed) {
#pragma unroll
    for (int f = 0; f < FG; ++f) {
      head[f] = tail[f];
      tail[f] = TR::zero();
    }
  }
}

// The total of output o = lane (lanes o < M): the tail of the lane whose
// chunk reaches into o from the previous output, then the heads of the
// lanes whose chunks start in o, in lane (that is, product) order.  At most
// ceil(32 / M) chunks start in one output; kFlatHeads bounds that for M >= 11.
constexpr int kFlatHeads = 3;
template <class TR>
__device__ __forceinline__ typename TR::Acc flat_combine(const typename TR::Acc& head, const typename TR::Acc& tail,
                                                         int M, int K, int lane) {
  using Acc = typename TR::Acc;
  const int W = M * K, c = (W + 31) >> 5;
  const int o = lane;
  const int la = (o * K + c - 1) / c;            // first lane starting in output o
  const int lb = ((o + 1) * K + c - 1) / c - 1;  // last lane starting in output o
  const Acc t = TR::shfl_idx(tail, max(la - 1, 0));
  Acc tot = (la >= 1 && la * c > o * K) ? t : TR::zero();
#pragma unroll
  for (int r = 0; r < kFlatHeads; ++r) {
    const Acc hv = TR::shfl_idx(head, min(la + r, 31));
    if (la + r <= lb) TR::merge(tot, hv);
  }
  return tot;
}

// Whether the flattened mapping costs fewer FP64 instructions for an op of
// M outputs and K inputs: c products per lane plus the combining adds,
// against ceil(K / ks) products per lane plus the reduction tree's adds.
__device__ __forceinline__ bool flat_pays(int M, int K, int ks) {
  if (M < 11 || M > 32) return false;
  const int tree = 2 * ((K + ks - 1) / ks) + (ks == 2 ? 2 : 0);
  const int flat = 2 * ((M * K + 31) >> 5) + 2 * (kFlatHeads + 1);
  return flat < tree;
}

// floor(32 / M) for M = 0..32, and ceil(65536 / d) for d = 0..32.
__constant__ unsigned char c_lanes_per_out[33] = {0, 32, 16, 10, 8, 6, 5, 4, 4, 3, 3, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
__constant__ unsigned c_inv16[33] = {0, 65536, 32768, 21846, 16384, 13108, 10923, 9363, 8192, 7282, 6554, 5958, 5462, 5042, 4682, 4370, 4096, 3856, 3641, 3450, 3277, 3121, 2979, 2850, 2731, 2622, 2521, 2428, 2341, 2260, 2185, 2115, 2048};

// What an op needs of its field: the launch's own arguments, or one field
// of a batched launch.
// What an op needs of its fields: the launch's own arguments (one field), or
// one group of a batched launch (nf fields sharing a plan, whose inputs and
// outputs come from the device pointer arrays, listed by group_fields).
template <int FG>
struct FieldCtx {
  const uint8_t* values;
  const void* in[FG];
  void* out[FG];
  const double* prescale;
  const double2* twiddle;
  int l;
  int nf;
  int buf_ab;
  int plain;  // single-block I/O (SweepArgs::plain)
};
template <int FG>
__device__ __forceinline__ FieldCtx<FG> field_ctx(const SweepArgs& A, int g) {
  FieldCtx<FG> c;
  c.plain = A.plain;
  if (!A.fields) {
    c.values = A.values;
    c.prescale = A.prescale;
    c.twiddle = A.twiddle;
    c.l = A.l;
    c.nf = 1;
    c.buf_ab = A.buf_ab;
#pragma unroll
    for (int f = 0; f < FG; ++f) {
      c.in[f] = A.in;
      c.out[f] = A.out;
    }
    return c;
  }
  const FieldDesc& d = A.fields[g];
  c.values = d.values;
  c.prescale = d.prescale;
  c.twiddle = d.twiddle;
  c.l = d.l;
  c.nf = min(d.nf, FG);
  c.buf_ab = d.buf_ab;
#pragma unroll
  for (int f = 0; f < FG; ++f) {
    const int k = A.group_fields[d.f0 + (f < c.nf ? f : 0)];
    c.in[f] = A.field_in[k];
    c.out[f] = A.field_out[k];
  }
  return c;
}

// One compute op (SYN_INTERP, DENSE, DENSE_G, ANA_INTERP), executed by one
// warp for every field of the item's group.
template <class TR, int FG, class AfterRead>
__device__ __forceinline__ void run_gemv(const OpHdr& h, const uint8_t* op, const Vecs<TR>& S,
                                         const FieldCtx<FG>& A, int lane, const uint8_t* staged,
                                         AfterRead after_read) {
  using C = typename TR::C;
  using V = typename TR::V;
  using Acc = typename TR::Acc;
  using IO = typename TR::IO;
  const int M = h.M, K = h.K;
  const int nf = A.nf;
  const uint16_t* idx = reinterpret_cast<const uint16_t*>(op + sizeof(OpHdr)) + h.npred;
  const V* val = reinterpret_cast<const V*>(staged);  // this warp's staging slot
  const bool gather = (h.kind == OP_SYN_INTERP);
  const bool accum = (h.flags & F_ACCUM) != 0;
  // vector positions: 16 bits, plus the bits above in a1 for single blocks
  const int io = h.io + (A.plain ? (int)(h.a1 & 0xFFFFu) << 16 : 0);
  const int oo = h.oo + (A.plain ? (int)(h.a1 >> 16) << 16 : 0);
  if (M > 0) {
    // stores output o of field f from its total a0 (the lane that owns o)
    auto store = [&](int f, Acc a0, int o) {
      const C* in = S.buf(h.in_buf, f) + io;
      C* out = S.buf(h.out_buf, f) + oo;
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
          const int i = oo + o;
          IO v = TR::to_io(TR::to_c(a0));
          if (A.plain) {  // node value i of a single block
            IO* y = reinterpret_cast<IO*>(A.out[f]);
            y[i] = accum ? TR::io_add(y[i], v) : v;
            break;
          }
          if (A.twiddle) v = TR::io_cmul(v, A.twiddle[h.a1]);
          IO* G = reinterpret_cast<IO*>(A.out[f]) + (size_t)h.a1 * (2 * l);
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
    };
    // ks = floor(32 / M) lanes per output (not only powers of two, so that
    // up to 32 - ks + 1 lanes work); lane = o * ks + q.  Both divisions come
    // from a table: lane / ks = (lane * ceil(2^16 / ks)) >> 16 holds exactly
    // for lane < 32 and ks <= 32.
    const int ks = c_lanes_per_out[M];
    if constexpr (TR::kSplitComponents) {
      // float64 ops whose outputs leave lanes idle: the flattened mapping
      if (flat_pays(M, K, ks)) {
        const C* inp[FG];
#pragma unroll
        for (int f = 0; f < FG; ++f) inp[f] = S.buf(h.in_buf, f) + io;
        Acc head[FG], tail[FG];
        flat_dot<TR, FG>(val, inp, idx, gather, M, K, lane, nf, head, tail);
        after_read();  // every lane is done with the staged values
#pragma unroll
        for (int f = 0; f < FG; ++f) {
          if (f >= nf) break;
          const Acc a0 = flat_combine<TR>(head[f], tail[f], M, K, lane);
          if (lane < M) store(f, a0, lane);
        }
        goto skel;
      }
    }
    {
    const int o = (lane * c_inv16[ks]) >> 16, q = lane - o * ks;
    Acc a[FG];
    if constexpr (FG == 1) {
      a[0] = TR::zero();
      if (o < M) a[0] = gemv_dot<TR>(val, S.buf(h.in_buf) + io, idx, gather, M, K, o, q, ks);
    } else {
      const C* inp[FG];
#pragma unroll
      for (int f = 0; f < FG; ++f) inp[f] = S.buf(h.in_buf, f) + io;
      if (o < M) {
        gemv_dot_fields<TR, FG>(val, inp, idx, gather, M, K, o, q, ks, nf, a);
      } else {
#pragma unroll
        for (int f = 0; f < FG; ++f) a[f] = TR::zero();
      }
    }
    after_read();  // every lane is done with the staged values
#pragma unroll
    for (int f = 0; f < FG; ++f) {
      if (f >= nf) break;
      Acc a0 = a[f];
      if constexpr (TR::kSplitComponents) {
        if (ks >= 2 && (ks & (ks - 1)) == 0) {
          // float64, ks a power of two: the same tree with the components
          // split between lane pairs.  Lanes q and q ^ 1 first exchange one
          // component each, so that even lanes carry the real sums and odd
          // lanes the imaginary ones; every further step adds one double
          // instead of two (the FP64 pipe is the bound).  Each sum is the
          // plain tree's, operand for operand, so the results are the same
          // bits.  Lane q = 0 ends with the real part, q = 1 with the
          // imaginary part.
          const int comp = q & 1;
          double v = comp ? a0.im : a0.re;
          const double give = comp ? a0.re : a0.im;
          v += __shfl_xor_sync(0xffffffffu, give, 1);
          for (int off = 2; off < ks; off <<= 1) {
            const double b = __shfl_down_sync(0xffffffffu, v, off);
            if (q + off < ks) v += b;
          }
          if (h.kind == OP_DENSE_G && A.twiddle && !A.plain) {
            // the phase mixes the components: lane q = 0 takes both
            const double w = __shfl_xor_sync(0xffffffffu, v, 1);
            if (q == 0 && o < M) {
              const int l = A.l;
              const int i = oo + o;
              IO z = TR::io_cmul(make_double2(v, w), A.twiddle[h.a1]);
              IO* G = reinterpret_cast<IO*>(A.out[f]) + (size_t)h.a1 * (2 * l);
              if (accum) {
                G[l + i] = TR::io_add(G[l + i], z);
                G[l - 1 - i] = TR::io_sub(G[l - 1 - i], z);
              } else {
                G[l + i] = z;
                G[l - 1 - i] = z;
              }
            }
          } else if (q < 2 && o < M) {
            const double* in = reinterpret_cast<const double*>(S.buf(h.in_buf, f) + io);
            double* out = reinterpret_cast<double*>(S.buf(h.out_buf, f) + oo);
            switch (h.kind) {
              case OP_SYN_INTERP:
                out[2 * o + comp] = v + in[2 * idx[K + o] + comp];
                break;
              case OP_DENSE:
                out[2 * o + comp] = v;
                break;
              case OP_ANA_INTERP: {
                const int pos = idx[o];
                out[2 * pos + comp] = accum ? v + out[2 * pos + comp] : v;
                break;
              }
              case OP_DENSE_G: {
                const int l = A.l;
                const int i = oo + o;
                if (A.plain) {
                  double* y = reinterpret_cast<double*>(A.out[f]);
                  y[2 * i + comp] = accum ? y[2 * i + comp] + v : v;
                  break;
                }
                double* G = reinterpret_cast<double*>(reinterpret_cast<IO*>(A.out[f]) + (size_t)h.a1 * (2 * l));
                if (accum) {
                  G[2 * (l + i) + comp] = G[2 * (l + i) + comp] + v;
                  G[2 * (l - 1 - i) + comp] = G[2 * (l - 1 - i) + comp] - v;
                } else {
                  G[2 * (l + i) + comp] = v;
                  G[2 * (l - 1 - i) + comp] = v;
                }
                break;
              }
              default:
                break;
            }
          }
          continue;
        }
      }
      // segmented tree: after the step with offset d, lane q holds the sum
      // over q .. min(q + 2d - 1, ks - 1) of its segment
      for (int off = 1; off < ks; off <<= 1) {
        const Acc b = TR::shfl_down(a0, off);
        if (q + off < ks) TR::merge(a0, b);
      }
      if (q == 0 && o < M) store(f, a0, o);
    }
    }
  }
skel:
  if (h.kind == OP_ANA_INTERP && (h.flags & F_SKEL)) {
    const uint16_t* skel = idx + M;
    for (int f = 0; f < nf; ++f) {
      const C* in = S.buf(h.in_buf, f) + io;
      C* out = S.buf(h.out_buf, f) + oo;
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
}

// One control op over the element range [oo, oo + M), executed by one warp
// for every field of the item's group.
template <class TR, int FG>
__device__ __forceinline__ void run_control(const OpHdr& h, const Vecs<TR>& S, const FieldCtx<FG>& A, int lane) {
  using C = typename TR::C;
  using IO = typename TR::IO;
  const int l = A.l, L = 2 * l;
  const int m = (int)h.a1;
  const int n = h.M;
  const int parity = h.a0 & 1, base = h.a0 >> 1;  // GATHER / SCATTER / FOLD
  // element offsets: 16 bits, plus the bits above in a1 for single blocks
  // (only a clear of a level vector needs them there)
  const int io = h.io + (A.plain ? (int)(h.a1 & 0xFFFFu) << 16 : 0);
  const int oo = h.oo + (A.plain ? (int)(h.a1 >> 16) << 16 : 0);
  // coefficient j of this parity: element 2j of order m's triangle row, or
  // element j of a plain vector (single blocks)
  const size_t c0 = A.plain ? 0 : tri_off(m, L) + parity;
  const int cs = A.plain ? 1 : 2;
  for (int f = 0; f < A.nf; ++f) {
    switch (h.kind) {
      case OP_GATHER: {
        const IO* beta = reinterpret_cast<const IO*>(A.in[f]) + c0;
        C* dst = S.buf(h.out_buf, f) + base;
        for (int j = oo + lane; j < oo + n; j += 32) dst[j] = TR::from_io(beta[cs * (size_t)j]);
        break;
      }
      case OP_SCATTER: {
        IO* beta = reinterpret_cast<IO*>(A.out[f]) + c0;
        const C* src = S.buf(h.in_buf, f) + base;
        for (int j = io + lane; j < io + n; j += 32) beta[cs * (size_t)j] = TR::to_io(src[j]);
        break;
      }
      case OP_FOLD: {
        const IO* G = reinterpret_cast<const IO*>(A.in[f]) + (A.plain ? 0 : (size_t)m * L);
        C* dst = S.buf(h.out_buf, f) + base;
        for (int r = oo + lane; r < oo + n; r += 32) {
          IO e;
          if (A.plain) {
            e = G[r];  // node value r of a single block: nothing to fold
          } else {
            IO gp = G[l + r], gm = G[l - 1 - r];
            if (A.twiddle) {
              gp = TR::io_cmul(gp, A.twiddle[m]);
              gm = TR::io_cmul(gm, A.twiddle[m]);
            }
            e = parity ? TR::io_sub(gp, gm) : TR::io_add(gp, gm);
          }
          if (A.prescale) e = TR::io_scale(e, A.prescale[r]);
          dst[r] = TR::from_io(e);
        }
        break;
      }
      case OP_CLEAR: {
        C* dst = S.buf(h.out_buf, f);
        for (int j = oo + lane; j < oo + n; j += 32) dst[j] = TR::czero();
        break;
      }
      case OP_GZERO: {
        if (A.plain) {
          IO* y = reinterpret_cast<IO*>(A.out[f]);
          for (int r = oo + lane; r < oo + n; r += 32) y[r] = TR::io_zero();
          break;
        }
        IO* G = reinterpret_cast<IO*>(A.out[f]) + (size_t)m * L;
        for (int r = oo + lane; r < oo + n; r += 32) {
          G[l + r] = TR::io_zero();
          G[l - 1 - r] = TR::io_zero();
        }
        break;
      }
      default:
        break;
    }
  }
}


// ------------------------------------------------------------ warps

__device__ __forceinline__ unsigned vload(const unsigned* p) { return *reinterpret_cast<const volatile unsigned*>(p); }
__device__ __forceinline__ void vstore(unsigned* p, unsigned v) { *reinterpret_cast<volatile unsigned*>(p) = v; }

// Shared control words of one CTA.
struct Ctl {
  unsigned progress[kMaxWarps];  // warp w has completed ops 0..n-1 of item seq: seq * 4096 + n
  unsigned item[2];              // number of item seq at [seq & 1] (>= n_units: the queue is empty)
  unsigned arrived;              // warps that finished their part of items 0..seq: NW * (seq + 1)
  unsigned abort;                // set when a bounded wait gave up or a stream was refused
};

__device__ __forceinline__ void trace_add(const SweepArgs& A, int slot, unsigned long long v) {
  if (A.trace && v) atomicAdd(A.trace + slot, v);
}

// Records the error (first one wins) and stops the CTA.
__device__ __forceinline__ void fail(const SweepArgs& A, Ctl* S, unsigned code) {
  atomicCAS(A.status, 0u, code);
  vstore(&S->abort, 1u);
}

// Lane 0 polls until pred() holds (bounded; the CTA abort flag ends it too),
// then the warp agrees on the outcome and acquires what was published.
template <class Pred>
__device__ __forceinline__ bool warp_wait(Pred pred, const SweepArgs& A, Ctl* S, int lane) {
  int ok = 1;
  if (lane == 0 && !pred()) {
    const long long t0 = clock64();
    for (unsigned ns = 32;;) {
      __nanosleep(ns);
      if (pred()) break;
      if (vload(&S->abort)) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > kTimeoutCycles) {
        fail(A, S, kStatusTimeout);
        ok = 0;
        break;
      }
      ns = ns < 256 ? 2 * ns : 256;
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __threadfence_block();
  return ok != 0;
}

// Every lane polls the mbarrier phase itself, so each lane's successful
// try_wait is its own acquire of the copied bytes; bounded like warp_wait.
__device__ __forceinline__ bool warp_poll_mbar(uint64_t* bar, uint32_t parity, const SweepArgs& A, Ctl* S,
                                               int lane) {
  if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
  const long long t0 = clock64();
  for (;;) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    int bad = 0;
    if (lane == 0) {
      if (vload(&S->abort)) {
        bad = 1;
      } else if (clock64() - t0 > kTimeoutCycles) {
        fail(A, S, kStatusTimeout);
        bad = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, bad, 0)) return false;
  }
}

// One warp's walk over its scheduled ops of every item its CTA takes.
template <class TR, int NW, int FG>
__device__ void warp_loop(const SweepArgs& A, Ctl* S, typename TR::C* vec_base, int warp, int lane, uint8_t* ring,
                          uint64_t* ring_bar, uint8_t* slot, uint64_t* slot_bar) {
  using Val = typename TR::V;
  const uint32_t CH = (uint32_t)A.chunk_bytes;  // a power of two
  const uint32_t csh = (uint32_t)(__ffs(A.chunk_bytes) - 1);
  const bool tracing = A.trace != nullptr;
  unsigned long long c_gemv = 0, c_ctl = 0, c_dep = 0, c_val = 0, c_rec = 0, c_bar = 0, c_done = 0;
  unsigned long long n_gemv = 0, n_ctl = 0, n_items = 0;
  uint32_t ring_par = 0;   // bit r: parity of ring slot r's next completion
  uint32_t ring_busy = 0;  // bit r: a copy into ring slot r has not been waited for
  uint32_t slot_par = 0;   // parity of the staging slot's next completion
  bool slot_busy = false;  // a copy into the staging slot has not been waited for

  for (unsigned seq = 0;; ++seq) {
    const unsigned item = vload(&S->item[seq & 1]);
    if (item >= (unsigned)A.n_units || vload(&S->abort)) break;
    if (warp == 0 && lane == 0) {
      // the next item's number, fetched while this one runs; the CTA that
      // takes the last number past the end resets the queue for the next launch
      const unsigned u = atomicAdd(A.counter, 1u);
      if (u == (unsigned)A.n_units + gridDim.x - 1) atomicExch(A.counter, 0u);
      vstore(&S->item[(seq + 1) & 1], u);
    }
    const UnitEntry e = A.units[item];
    const int field = A.fields ? (int)e.m : 0;  // batched launches: the item's field group
    const FieldCtx<FG> F = field_ctx<FG>(A, field);
    const Vecs<TR> V{vec_base, F.buf_ab};
    const uint8_t* region = A.fields ? A.fields[field].pages : A.pages;
    const uint8_t* item_base = region + e.off16 * 16;
    // this warp's record stream; a stream scheduled for another warp count,
    // or a batched field with a bad input or output pointer, is refused
    uint32_t off = 0, len = 0;
    if (lane == 0) {
      const ItemHeader ih = *reinterpret_cast<const ItemHeader*>(item_base);
      const WarpRange wr = reinterpret_cast<const WarpRange*>(item_base + sizeof(ItemHeader))[warp];
      bool bad = ih.magic != kItemMagic || ih.nw != NW || (wr.off & 15u) || (wr.bytes & 15u) ||
                 (uint64_t)wr.off + wr.bytes > (uint64_t)e.len16 * 16;
      if (A.fields)
        for (int f = 0; f < F.nf; ++f) {
          const uintptr_t io = reinterpret_cast<uintptr_t>(F.in[f]) | reinterpret_cast<uintptr_t>(F.out[f]);
          bad = bad || !F.in[f] || !F.out[f] || (io & (uintptr_t)(A.io_align - 1));
        }
      if (bad) fail(A, S, kStatusBadArg);
      off = bad ? 0 : wr.off;
      len = bad ? 0 : wr.bytes;
    }
    off = __shfl_sync(0xffffffffu, off, 0);
    len = __shfl_sync(0xffffffffu, len, 0);
    const uint8_t* stream = item_base + off;
    const uint32_t nch = (len + CH - 1) >> csh;
    auto issue_chunk = [&](uint32_t c) {  // lane 0; chunk c into ring slot c & 1
      const uint32_t r = c & 1u;
      const uint32_t bytes = min(CH, len - c * CH);
      fence_proxy_async();  // earlier reads of the slot precede the copy into it
      mbar_arrive_expect_tx(ring_bar + r, bytes);
      bulk_g2s(ring + (size_t)r * CH, stream + (size_t)c * CH, bytes, ring_bar + r);
    };
    if (lane == 0)
      for (uint32_t c = 0; c < nch && c < 2; ++c) issue_chunk(c);
    ring_busy |= (nch > 0 ? 1u : 0u) | (nch > 1 ? 2u : 0u);
    auto has_values = [](const OpHdr& h) {
      return h.kind >= OP_SYN_INTERP && h.kind <= OP_ANA_INTERP && h.M > 0 && h.K > 0;
    };
    // a compute op must fit one warp and its values the staging slot
    auto sound = [&](const OpHdr& h) {
      const bool g = h.kind >= OP_SYN_INTERP && h.kind <= OP_ANA_INTERP;
      return !g || (h.M <= kMaxM && sizeof(Val) * h.M * h.K <= (size_t)A.slot_bytes);
    };
    auto issue_values = [&](const OpHdr& h) {  // lane 0, for a sound op with values
      const uint32_t vb = (uint32_t)((sizeof(Val) * h.M * h.K + 15) & ~size_t(15));
      fence_proxy_async();
      mbar_arrive_expect_tx(slot_bar, vb);
      bulk_g2s(slot, F.values + (size_t)h.vref * 16, vb, slot_bar);
    };
    // Waits for chunk c (all lanes acquire its bytes); false if aborted.
    uint32_t waited = 0;  // chunks waited for so far
    auto wait_chunk = [&](uint32_t c) -> bool {
      for (; waited <= c; ++waited) {
        const uint32_t r = waited & 1u;
        const uint32_t ph = (ring_par >> r) & 1u;
        const long long t0 = tracing ? clock64() : 0;
        if (!warp_poll_mbar(ring_bar + r, ph, A, S, lane)) return false;
        ring_par ^= 1u << r;
        ring_busy &= ~(1u << r);
        if (tracing) c_rec += clock64() - t0;
      }
      return true;
    };
    bool ok = true;
    uint32_t pending = 0xffffffffu;  // position of the value op whose block the staging slot receives
    uint32_t n_done = 0, cur_c = 0;  // cur_c: chunk of the last record run
    // Finds the record at or after position np (skipping a chunk's padding,
    // waiting for its chunk): its position and header, or false at the end.
    auto peek = [&](uint32_t np, uint32_t& at, OpHdr& nh) -> bool {
      while (np < len) {
        const uint32_t cn = np >> csh, in = np & (CH - 1);
        if (in + sizeof(OpHdr) > CH) {  // too little room left for a record: padding
          np = (cn + 1) << csh;
          continue;
        }
        if (!wait_chunk(cn)) return false;
        nh = *reinterpret_cast<const OpHdr*>(ring + ((size_t)(cn & 1u) << csh) + in);
        if (nh.bytes == 0) {
          np = (cn + 1) << csh;
          continue;
        }
        at = np;
        return true;
      }
      return false;
    };
    uint32_t rpos = 0;
    OpHdr h;
    bool have = peek(0, rpos, h);
    while (have && ok) {
      const uint32_t c = rpos >> csh, in = rpos & (CH - 1);
      // chunks before this record's are used up: refill their ring slots
      for (uint32_t cf = cur_c; cf < c; ++cf) {
        __syncwarp();
        if (lane == 0 && cf + 2 < nch) issue_chunk(cf + 2);
        if (cf + 2 < nch) ring_busy |= 1u << (cf & 1u);
      }
      cur_c = c;
      const uint8_t* rec = ring + ((size_t)(c & 1u) << csh) + in;
      // a record must lie in its chunk, and a compute op fit one warp and
      // its values the staging slot (what keeps every access in bounds)
      if (in + h.bytes > CH || !sound(h)) {
        if (lane == 0) fail(A, S, kStatusBadArg);
        ok = false;
        break;
      }
      const bool gemv = h.kind >= OP_SYN_INTERP && h.kind <= OP_ANA_INTERP;
      const bool vals = has_values(h);
      if (vals && pending != rpos) {  // not prefetched by the previous op
        if (lane == 0) issue_values(h);
        slot_busy = true;
        pending = rpos;
      }
      // the next record: its values are copied into the slot as soon as this
      // op has read it (at once if this op has no values)
      uint32_t nat = 0;
      OpHdr nh;
      const bool have_next = peek(rpos + h.bytes, nat, nh);  // false also if the CTA gave up
      const bool next_vals = have_next && has_values(nh) && sound(nh);
      auto prefetch = [&]() {
        if (next_vals && pending != nat) {
          __syncwarp();
          if (lane == 0) issue_values(nh);
          slot_busy = true;
          pending = nat;
        }
      };
      if (!vals && !slot_busy) prefetch();
      // wait for the listed warps' progress
      const long long t1 = tracing ? clock64() : 0;
      if (h.npred) {
        const uint16_t* pred = reinterpret_cast<const uint16_t*>(rec + sizeof(OpHdr));
        unsigned want_w = 0, want = 0;
        const bool mine = lane < h.npred;
        if (mine) {
          const unsigned ent = pred[lane];
          want_w = ent >> kPredPosBits;
          want = seq * 4096u + (ent & ((1u << kPredPosBits) - 1)) + 1u;
        }
        auto met = [&] { return !mine || vload(&S->progress[want_w]) >= want; };
        if (!__all_sync(0xffffffffu, met())) {
          const long long t0 = clock64();
          for (unsigned ns = 32;;) {
            __nanosleep(ns);
            if (__all_sync(0xffffffffu, met())) break;
            int bad = 0;
            if (lane == 0) {
              if (vload(&S->abort)) {
                bad = 1;
              } else if (clock64() - t0 > kTimeoutCycles) {
                fail(A, S, kStatusTimeout);
                bad = 1;
              }
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) {
              ok = false;
              break;
            }
            ns = ns < 128 ? 2 * ns : 128;
          }
        }
        __threadfence_block();  // acquire what the predecessors wrote
        if (!ok) break;
      }
      const long long t2 = tracing ? clock64() : 0;
      if (vals) {
        if (!warp_poll_mbar(slot_bar, slot_par, A, S, lane)) {
          ok = false;
          break;
        }
        slot_par ^= 1u;
        slot_busy = false;
      }
      const long long t3 = tracing ? clock64() : 0;
      if (gemv) {
        run_gemv<TR, FG>(h, rec, V, F, lane, slot, [&] {
          if (!slot_busy) prefetch();
        });
      } else {
        run_control<TR, FG>(h, V, F, lane);
      }
      if (!slot_busy) prefetch();  // ops without a value block
      const long long t4 = tracing ? clock64() : 0;
      ++n_done;
      if (h.flags & F_PUBLISH) {  // another warp waits for this op: publish
        __threadfence_block();
        __syncwarp();
        if (lane == 0) vstore(&S->progress[warp], seq * 4096u + n_done);
      }
      if (tracing) {
        const long long t5 = clock64();
        if (gemv) {
          c_gemv += t4 - t3;
          ++n_gemv;
        } else {
          c_ctl += t4 - t3;
          ++n_ctl;
        }
        c_dep += t2 - t1;
        c_val += t3 - t2;
        c_done += t5 - t4;
      }
      rpos = nat;
      h = nh;
      have = have_next;
    }
    if (!ok) break;
    // every warp has finished this item before any starts the next
    const long long tb = tracing ? clock64() : 0;
    __threadfence_block();  // this warp's writes of the item precede its arrival
    __syncwarp();
    if (lane == 0) atomicAdd(&S->arrived, 1u);
    if (!warp_wait([&] { return vload(&S->arrived) >= (unsigned)NW * (seq + 1); }, A, S, lane)) break;
    if (tracing) {
      c_bar += clock64() - tb;
      ++n_items;
    }
  }
  // never leave with a bulk copy still landing in this warp's ring or slot
  if (lane == 0) {
    for (uint32_t r = 0; r < 2; ++r)
      if ((ring_busy >> r) & 1u) wait_bounded(ring_bar + r, (ring_par >> r) & 1u, A.status, (volatile int*)&S->abort);
    if (slot_busy) wait_bounded(slot_bar, slot_par, A.status, (volatile int*)&S->abort);
  }
  __syncwarp();
  if (lane == 0 && tracing) {
    trace_add(A, TR_EXEC_GEMV, c_gemv);
    trace_add(A, TR_EXEC_CTL, c_ctl);
    trace_add(A, TR_WAIT_DEP, c_dep);
    trace_add(A, TR_WAIT_VALUES, c_val);
    trace_add(A, TR_WAIT_RECORDS, c_rec);
    trace_add(A, TR_WAIT_BARRIER, c_bar);
    trace_add(A, TR_N_GEMV, n_gemv);
    trace_add(A, TR_N_CTL, n_ctl);
    trace_add(A, TR_N_ITEMS, n_items);
    trace_add(A, TR_COMPLETE, c_done);
  }
}

// Shared-memory layout of a sweep CTA, used by the kernel and by the host
// sizing alike: | vectors (128-aligned; none when they are in global memory)
// | per warp: two record chunks, the staging slot | mbarriers: per warp two
// ring + one slot (+1 spare) | Ctl |.
__host__ __device__ inline size_t sweep_vec_bytes(size_t c_size, int num_vecs, int buf_ab) {
  return (c_size * (size_t)num_vecs * (size_t)buf_ab + 127) & ~size_t(127);
}
__host__ __device__ inline size_t sweep_warp_bytes(int chunk_bytes, int slot_bytes) {
  return (2 * (size_t)chunk_bytes + (size_t)slot_bytes + 127) & ~size_t(127);
}

template <class TR, int NW, int FG>
__global__ void __launch_bounds__(NW * 32, 1) bfly_sweep_kernel(const SweepArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // vectors in shared memory, or in global memory for the whole launch
  const size_t vec_bytes = A.gvec ? 0 : sweep_vec_bytes(sizeof(typename TR::C), A.num_vecs, A.buf_ab);
  const size_t wb = sweep_warp_bytes(A.chunk_bytes, A.slot_bytes);
  uint8_t* mine = smem + vec_bytes + (size_t)warp * wb;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + vec_bytes + (size_t)NW * wb);
  Ctl* S = reinterpret_cast<Ctl*>(bars + 4 * NW);

  if (tid == 0) {
    for (int s = 0; s < 4 * NW; ++s) mbar_init(bars + s, 1);
    for (int w = 0; w < kMaxWarps; ++w) S->progress[w] = 0;
    S->arrived = 0;
    S->abort = 0;
    const unsigned u = atomicAdd(A.counter, 1u);
    if (u == (unsigned)A.n_units + gridDim.x - 1) atomicExch(A.counter, 0u);
    S->item[0] = u;
    S->item[1] = 0xffffffffu;
    fence_mbar_init();
  }
  __syncthreads();
  typename TR::C* vecs = A.gvec ? reinterpret_cast<typename TR::C*>(A.gvec) : reinterpret_cast<typename TR::C*>(smem);
  warp_loop<TR, NW, FG>(A, S, vecs, warp, lane, mine, bars + 4 * warp,
                        mine + 2 * (size_t)A.chunk_bytes, bars + 4 * warp + 2);
}

template <class TR>
size_t smem_for(int chunk_bytes, int buf_ab, int num_vecs, int nw, int slot_bytes) {
  return sweep_vec_bytes(sizeof(typename TR::C), num_vecs, buf_ab) + (size_t)nw * sweep_warp_bytes(chunk_bytes, slot_bytes) +
         sizeof(uint64_t) * 4 * (size_t)nw + sizeof(Ctl);
}

}  // namespace

size_t sweep_smem_bytes(int prec, int chunk_bytes, int buf_ab, int num_vecs, int nw, int slot_bytes, int warp_slots) {
  (void)warp_slots;  // one staging slot per warp
  switch (prec) {
    case PREC_FP64: return smem_for<TF64>(chunk_bytes, buf_ab, num_vecs, nw, slot_bytes);
    case PREC_FP32: return smem_for<TF32>(chunk_bytes, buf_ab, num_vecs, nw, slot_bytes);
    case PREC_SPLIT32_ACC64: return smem_for<TS32A>(chunk_bytes, buf_ab, num_vecs, nw, slot_bytes);
    default: return smem_for<TS32>(chunk_bytes, buf_ab, num_vecs, nw, slot_bytes);
  }
}

namespace {

// Host dispatch over (precision, consumer warps, fields per group); groups
// of 2 or 4 fields run with 16 warps only.
template <class TR>
const void* kernel_ptr(int nw, int fg) {
  if (nw == 16 && fg == 4) return reinterpret_cast<const void*>(bfly_sweep_kernel<TR, 16, 4>);
  if (nw == 16 && fg == 2) return reinterpret_cast<const void*>(bfly_sweep_kernel<TR, 16, 2>);
  switch (nw) {
    case 8: return reinterpret_cast<const void*>(bfly_sweep_kernel<TR, 8, 1>);
    case 12: return reinterpret_cast<const void*>(bfly_sweep_kernel<TR, 12, 1>);
    default: return reinterpret_cast<const void*>(bfly_sweep_kernel<TR, 16, 1>);
  }
}
const void* kernel_for(int prec, int nw, int fg) {
  switch (prec) {
    case PREC_FP64: return kernel_ptr<TF64>(nw, fg);
    case PREC_FP32: return kernel_ptr<TF32>(nw, fg);
    case PREC_SPLIT32_ACC64: return kernel_ptr<TS32A>(nw, fg);
    default: return kernel_ptr<TS32>(nw, fg);
  }
}

}  // namespace

cudaError_t sweep_configure(int prec, size_t smem) {
  for (int nw : {8, 12, 16})
    for (int fg : {1, 2, 4}) {
      if (fg > 1 && nw != 16) continue;
      cudaError_t e =
          cudaFuncSetAttribute(kernel_for(prec, nw, fg), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

int sweep_blocks_per_sm(int prec, int nw, size_t smem) {
  int nb = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_for(prec, nw, 1), nw * 32, smem);
  return (e == cudaSuccess && nb > 0) ? nb : 1;
}

bool sweep_choose(int prec, int chunk_bytes, int buf_ab, int num_vecs, int nw, int slot_bytes, int warp_slots,
                  size_t optin, SweepConfig* c) {
  c->nw = nw;
  c->warp_slots = 1;
  (void)warp_slots;
  c->slot_bytes = slot_bytes;
  c->smem = sweep_smem_bytes(prec, chunk_bytes, buf_ab, num_vecs, nw, slot_bytes, 1);
  if (c->smem > optin) {
    c->ctas_per_sm = 0;
    return false;
  }
  c->ctas_per_sm = std::min(2, sweep_blocks_per_sm(prec, nw, c->smem));
  return true;
}

cudaError_t sweep_launch(int prec, int nw, const SweepArgs& a, int grid, size_t smem, cudaStream_t st) {
  if (nw != 8 && nw != 12 && nw != 16) return cudaErrorInvalidValue;
  if (a.chunk_bytes < kMinChunkBytes || a.chunk_bytes > kMaxChunkBytes || (a.chunk_bytes & 255)) return cudaErrorInvalidValue;
  if (a.slot_bytes <= 0 || (a.slot_bytes & 15)) return cudaErrorInvalidValue;
  if (a.fg != 1 && !(nw == 16 && (a.fg == 2 || a.fg == 4) && a.fields)) return cudaErrorInvalidValue;
  void* args[] = {const_cast<SweepArgs*>(&a)};
  return cudaLaunchKernel(kernel_for(prec, nw, a.fg), dim3(grid), dim3(nw * 32), args, smem, st);
}

}  // namespace sht
