// plan_device.cu -- the depth-first butterfly precomputation of Section 3 on
// the device.
//
// A persistent grid takes parity blocks A^{m,p} from a queue (largest
// first); one CTA builds one block at a time, exactly in the order of the
// host builder (plan_build.cpp):
//   1. columns come from the x^2 recurrence of Section 2.3 (eqs. c_rec,
//      d_rec, recurrence0, recurrence) with the exponent tracking of Section
//      4, one row per thread: first over all n columns for the row norms that
//      trimming needs, then leaf by leaf;
//   2. each interpolative decomposition (Section 2.1, eq. 2.1) is a
//      column-pivoted Householder QR (Remark QR_algorithm) run by one warp:
//      rows across the lanes, pivot search and norms by warp shuffles, the
//      dot products of four trailing columns reduced together; the CTA's
//      eight warps factor independent blocks at once;
//   3. leaves are built eight at a time, one per warp, and merged with the
//      same pairing as the host's depth-first build (Section 3): every round
//      merges all pairs of same-level groups at the top of the stack, whose
//      ID blocks (two per band) are again shared among the warps.  The stack
//      of skeleton columns lives in global scratch.
// Every ID block and every band of the top level is written as one record
// into an output arena; the host reads the records back, lays each unit out
// (finish_unit) and encodes the streams as after a host build.  Nothing here
// waits on another CTA: the only synchronisation is __syncthreads.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "plan_host.h"
#include "recurrence.h"

namespace sht {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxGroups = 24;
constexpr int kBatch = kWarps;  // leaves factored at once, one per warp
constexpr unsigned kFull = 0xffffffffu;

enum UnitStatus { kPending = 0, kDone = 1, kNoArena = 2, kNoScratch = 3 };

// One record of the output arena (a multiple of 16 bytes).
//   kind 0, an ID block: header, int skel[k], int red[nin - k] (ascending),
//           padding to 16 bytes, double T[k * (nin - k)] (T[s * k + t]);
//   kind 1, a band of the top level: header, double S[(r1 - r0) * k].
struct RecHdr {
  int unit, kind, level, band, group, r0, r1, in_off, nin, k;
  long long bytes;
  int pad[4];
};
static_assert(sizeof(RecHdr) == 64, "record header size");

struct BandDesc {
  int r0, r1, k, pad;
  long long off;  // words into the CTA's stack
};
struct GroupDesc {
  int level, g, nb, d0;  // d0: first band descriptor
};

struct DevBuildArgs {
  int l, C, min_band_rows;
  double eps2;     // eps_id^2
  double trim2;    // (trim_eps / sqrt l)^2; 0: no trimming
  const double* xpos;  // x_{l+i}, i < l
  const double* spos;  // sin(theta_{l+i})
  const double* sq2w;  // sqrt(2 w_{l+i})
  const int* queue;    // unit ids u = 2m + p, largest first
  int n_queue;
  unsigned* next;      // queue counter
  double* scratch;     // per CTA: scratch_words
  long long scratch_words, buf_words, stack_words, desc_cap, warp_words;
  unsigned char* arena;
  unsigned long long arena_bytes;
  unsigned long long* arena_used;
  unsigned long long* arena_fail;  // lowest offset of a reservation that did not fit
  int* stop;                       // the arena is full: take no further units
  int* status;                     // per unit id
  long long* info;                 // per unit id: rows, levels, exchanges
};

struct Shared {
  GroupDesc grp[kMaxGroups];
  int redi[kWarps];
  int kres[kWarps];  // ranks of the leaves of the current batch
  unsigned long long tmp_sp;
  long long new_sp;
  int q, ngrp, ecm, fail, swaps;
  double cm;
};

__device__ __forceinline__ double warp_sum(double v) {
  // xor butterfly: every lane ends with the same bits (a + b == b + a)
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ int block_max_int(int v, Shared& S) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) S.redi[threadIdx.x >> 5] = v;
  __syncthreads();
  int r = S.redi[0];
#pragma unroll
  for (int i = 1; i < kWarps; ++i) r = max(r, S.redi[i]);
  return r;
}

__device__ __forceinline__ bool better(long long a, int ia, long long b, int ib) {
  return a > b || (a == b && ia < ib);
}

// Index of the largest x[j], i0 <= j < w, the lowest on ties (the host's
// pivot rule); i0 if there is none.  The x[j] are squared norms, never
// negative, so their bit patterns order like their values and the search
// runs on the integer pipes.  Every lane returns the same index.
__device__ __forceinline__ int warp_argmax(const double* x, int i0, int w, int lane) {
  long long best = -1;
  int bi = w;
  for (int j = i0 + lane; j < w; j += 32) {
    const long long b = __double_as_longlong(x[j]);
    if (b > best) {
      best = b;
      bi = j;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const long long ob = __shfl_xor_sync(kFull, best, o);
    const int oi = __shfl_xor_sync(kFull, bi, o);
    if (better(ob, oi, best, bi)) {
      best = ob;
      bi = oi;
    }
  }
  return bi < w ? bi : i0;
}

// Warp sums of four per-lane partial sums at once: each butterfly step
// halves the values a lane carries (column c ends in lanes 16 (c >> 1) +
// 8 (c & 1) + 0..7, all with the same bits), then every lane gets all four.
__device__ __forceinline__ void reduce4(double& d0, double& d1, double& d2, double& d3, int lane) {
  const bool hi16 = (lane & 16) != 0;
  double k0 = hi16 ? d2 : d0, k1 = hi16 ? d3 : d1;
  k0 += __shfl_xor_sync(kFull, hi16 ? d0 : d2, 16);
  k1 += __shfl_xor_sync(kFull, hi16 ? d1 : d3, 16);
  const bool hi8 = (lane & 8) != 0;
  double s = hi8 ? k1 : k0;
  s += __shfl_xor_sync(kFull, hi8 ? k0 : k1, 8);
#pragma unroll
  for (int o = 4; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  d0 = __shfl_sync(kFull, s, 0);
  d1 = __shfl_sync(kFull, s, 8);
  d2 = __shfl_sync(kFull, s, 16);
  d3 = __shfl_sync(kFull, s, 24);
}

// Warp sums of two per-lane partial sums (the first step splits them
// between the half-warps).
__device__ __forceinline__ void reduce2(double& x, double& y, int lane) {
  const bool hi16 = (lane & 16) != 0;
  double s = hi16 ? y : x;
  s += __shfl_xor_sync(kFull, hi16 ? x : y, 16);
#pragma unroll
  for (int o = 8; o; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  x = __shfl_sync(kFull, s, 0);
  y = __shfl_sync(kFull, s, 16);
}

__device__ __forceinline__ void renorm(double& v, int& e) {
  if (v == 0.0) return;
  int t;
  v = frexp(v, &t);
  e += t;
}

// Per-CTA views of the dynamic shared memory and the global scratch.
struct Views {
  // shared
  double *cinv, *cd, *cm2;  // per column j < n: 1/c_k, d_k, c_{k-2} (0 at j = 0), k = m + p + 2j
  // global, per CTA
  double *x2, *sqw, *ga, *gb;
  int* ge;
  BandDesc* desc;
  double* warps;  // kWarps x warp_words: each warp's Z, W, nrm, ref, perm
  long long warp_words;
  double* stack;
};

// One warp's buffers: the block Z (kept), its working copy W (destroyed by
// the QR), the squared column norms and the column order.
struct WarpBuf {
  double *Z, *W, *nrm, *ref;
  int* perm;
};
__device__ __forceinline__ WarpBuf warp_buf(const DevBuildArgs& A, const Views& V, int warp) {
  double* b = V.warps + (long long)warp * V.warp_words;
  WarpBuf B;
  B.Z = b;
  B.W = b + A.buf_words;
  B.nrm = B.W + A.buf_words;
  B.ref = B.nrm + A.l;
  B.perm = reinterpret_cast<int*>(B.ref + A.l);
  return B;
}

// Generator state of row i at column 0: b = P-bar^m_{m+p}(x_i) as a
// mantissa b and exponent e, a = 0 (eq. recurrence0 has no k - 2 term).
__device__ void row_init(const DevBuildArgs& A, const Shared& S, int m, int p, int i, double& x2, double& sqw,
                         double& a, double& b, int& e) {
  const double xi = A.xpos[i];
  x2 = xi * xi;
  sqw = A.sq2w[i];
  // sin(theta)^m by binary powering with tracked exponents
  int eb;
  double base = frexp(A.spos[i], &eb);
  double res = 1.0;
  int er = 0;
  for (int q = m; q; q >>= 1) {
    if (q & 1) {
      res *= base;
      er += eb;
      renorm(res, er);
    }
    base *= base;
    eb *= 2;
    renorm(base, eb);
  }
  double val = res * S.cm;
  int ev = er + S.ecm;
  if (p == 1) val *= sqrt(2.0 * m + 3.0) * xi;  // P-bar^m_{m+1} = sqrt(2m+3) x P-bar^m_m
  renorm(val, ev);
  a = 0.0;
  b = val;
  e = ev;
}

// Generator state of rows 0..rows-1 at column 0, kept in scratch.
__device__ void gen_init(const DevBuildArgs& A, const Views& V, const Shared& S, int m, int p, int rows) {
  for (int i = threadIdx.x; i < rows; i += kThreads)
    row_init(A, S, m, p, i, V.x2[i], V.sqw[i], V.ga[i], V.gb[i], V.ge[i]);
}

__device__ __forceinline__ int exp_field(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
// 2^k for -1022 <= k <= 1023, built from its bits
__device__ __forceinline__ double pow2(int k) { return __hiloint2double((k + 1023) << 20, 0); }

// One step of the recurrence for column j: returns the weighted value of
// column j and advances (a, b, e) to column j + 1.  The values are the host
// generator's bit for bit: products and sums are rounded one by one in its
// order; b 2^e is one product with an exact power of two where 2^e is a
// normal number (the same correctly rounded result as ldexp), and the
// rescaling test reads exponent fields, taking the host's exact rule
// whenever a value is near its thresholds (rescaling moves powers of two
// between (a, b) and e, which changes no later value).
__device__ __forceinline__ double gen_step(const Views& V, int j, double x2, double sqw, double& a, double& b,
                                           int& e) {
  const double be = ((unsigned)(e + 1022) <= 2045u) ? __dmul_rn(b, pow2(e)) : ldexp(b, e);
  const double col = __dmul_rn(sqw, be);
  const double nb = __dmul_rn(__dsub_rn(__dmul_rn(__dsub_rn(x2, V.cd[j]), b), __dmul_rn(V.cm2[j], a)), V.cinv[j]);
  a = b;
  b = nb;
  const int M = max(exp_field(a), exp_field(b));
  if (M >= 1023 + 400 || M < 1023 - 400) {
    const double big = fmax(fabs(a), fabs(b));
    if (big > 0x1p400 || (big < 0x1p-400 && big > 0.0)) {
      const int t = ilogb(big);
      a = ldexp(a, -t);
      b = ldexp(b, -t);
      e += t;
    }
  }
  return col;
}

// Columns of leaves g0 .. g0 + nb - 1 (consecutive column ranges), leaf
// g0 + q into warp q's Z (rows x width, column-major).
__device__ void gen_leaves(const DevBuildArgs& A, const Views& V, int g0, int nb, int nleaves, int n, int rows) {
  for (int i = threadIdx.x; i < rows; i += kThreads) {
    const double x2 = V.x2[i], sqw = V.sqw[i];
    double a = V.ga[i], b = V.gb[i];
    int e = V.ge[i];
    for (int q = 0; q < nb; ++q) {
      const int g = g0 + q;
      const int c0 = (int)((long long)g * n / nleaves), c1 = (int)((long long)(g + 1) * n / nleaves);
      double* out = warp_buf(A, V, q).Z;
      for (int j = c0; j < c1; ++j) out[(size_t)(j - c0) * rows + i] = gen_step(V, j, x2, sqw, a, b, e);
    }
    V.ga[i] = a;
    V.gb[i] = b;
    V.ge[i] = e;
  }
}

// Squared norms of rows r0.. of columns c0 .. w-1 into nrm and ref.
__device__ void warp_norms(const double* W, int h, int w, int c0, int r0, double* nrm, double* ref, int lane) {
  for (int j0 = c0; j0 < w; j0 += 4) {
    const int nc = min(4, w - j0);
    const double* c = W + (size_t)j0 * h;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    for (int r = r0 + lane; r < h; r += 32) {
      double x = c[r];
      d0 = fma(x, x, d0);
      if (nc > 1) {
        x = c[h + r];
        d1 = fma(x, x, d1);
      }
      if (nc > 2) {
        x = c[2 * h + r];
        d2 = fma(x, x, d2);
      }
      if (nc > 3) {
        x = c[3 * h + r];
        d3 = fma(x, x, d3);
      }
    }
    reduce4(d0, d1, d2, d3, lane);
    if (lane < nc) {
      const double s = lane == 0 ? d0 : lane == 1 ? d1 : lane == 2 ? d2 : d3;
      nrm[j0 + lane] = s;
      ref[j0 + lane] = s;
    }
  }
}

// Squared norm of column p's rows i.. (e) and rows i+1.. (sg).
__device__ __forceinline__ void pivot_sums(const double* W, int h, int p, int i, double& e, double& sg, int lane) {
  const double* c = W + (size_t)p * h;
  e = 0.0;
  sg = 0.0;
  for (int r = i + lane; r < h; r += 32) {
    const double x = c[r];
    e = fma(x, x, e);
    if (r > i) sg = fma(x, x, sg);
  }
  reduce2(e, sg, lane);
}

// Column-pivoted Householder QR of the h x w column-major W (destroyed) by
// one warp, to threshold eps2 on the squared residual column norms: the
// host's interp_decomp step for step.  Returns the rank k (every lane the
// same); perm holds the column order (skeleton first).  Within a step each
// lane owns the rows i+1+lane, i+33+lane, ...; __syncwarp separates steps
// and phases.
__device__ int warp_cpqr(double* W, int h, int w, double eps2, const WarpBuf& B, int lane) {
  double *nrm = B.nrm, *ref = B.ref;
  int* perm = B.perm;
  for (int j = lane; j < w; j += 32) perm[j] = j;
  warp_norms(W, h, w, 0, 0, nrm, ref, lane);
  __syncwarp();
  const int kmax = min(h, w);
  int k = 0;
  for (int i = 0; i < kmax; ++i) {
    int p = warp_argmax(nrm, i, w, lane);
    double e, sg;
    pivot_sums(W, h, p, i, e, sg, lane);
    if (e <= eps2) {
      // the downdated norms may have drifted: recompute all before stopping
      warp_norms(W, h, w, i, i, nrm, ref, lane);
      __syncwarp();
      p = warp_argmax(nrm, i, w, lane);
      if (nrm[p] <= eps2) break;
      pivot_sums(W, h, p, i, e, sg, lane);
    }
    // Householder reflector for the pivot column's rows i..
    const double alpha = W[(size_t)p * h + i];
    double tau = 0.0, beta = alpha, sc = 1.0;
    const bool reflect = (sg != 0.0 || alpha < 0.0);
    if (reflect) {
      const double nx = sqrt(alpha * alpha + sg);
      beta = (alpha <= 0.0) ? nx : -nx;
      tau = (beta - alpha) / beta;
      sc = 1.0 / (alpha - beta);
    }
    __syncwarp();  // alpha is read before row i is rewritten
    double* ci = W + (size_t)i * h;
    {
      double* cp = W + (size_t)p * h;
      for (int r = lane; r < h; r += 32) {
        const double t = cp[r], u = ci[r];
        double x = t;
        if (r == i) {
          x = beta;
        } else if (r > i && reflect) {
          x = t * sc;
        }
        if (p != i) cp[r] = u;
        ci[r] = x;
      }
      if (lane == 0) {
        nrm[p] = e;
        if (p != i) {
          const double tn = nrm[i], tr = ref[i];
          nrm[i] = nrm[p];
          ref[i] = ref[p];
          nrm[p] = tn;
          ref[p] = tr;
          const int tp = perm[i];
          perm[i] = perm[p];
          perm[p] = tp;
        }
      }
    }
    __syncwarp();
    // apply the reflector to the trailing columns, four at a time, and
    // downdate their norms
    for (int j0 = i + 1; j0 < w; j0 += 4) {
      const int nc = min(4, w - j0);
      double* c0 = W + (size_t)j0 * h;
      double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
      if (tau != 0.0) {
        for (int r = i + 1 + lane; r < h; r += 32) {
          const double vr = ci[r];
          d0 = fma(vr, c0[r], d0);
          if (nc > 1) d1 = fma(vr, c0[h + r], d1);
          if (nc > 2) d2 = fma(vr, c0[2 * h + r], d2);
          if (nc > 3) d3 = fma(vr, c0[3 * h + r], d3);
        }
        reduce4(d0, d1, d2, d3, lane);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c >= nc) break;
        const int j = j0 + c;
        double* cj = c0 + (size_t)c * h;
        double rij = cj[i];
        if (tau != 0.0) {
          const double dc = c == 0 ? d0 : c == 1 ? d1 : c == 2 ? d2 : d3;
          const double d = (dc + rij) * tau;
          for (int r = i + 1 + lane; r < h; r += 32) cj[r] = fma(-d, ci[r], cj[r]);
          rij -= d;
        }
        double nj = nrm[j] - rij * rij;
        const bool exact = nj < 1e-4 * ref[j];
        if (exact) {
          double s2 = 0.0;
          for (int r = i + 1 + lane; r < h; r += 32) s2 = fma(cj[r], cj[r], s2);
          nj = warp_sum(s2);
        }
        __syncwarp();  // every lane has read cj[i], nrm[j] and ref[j]
        if (lane == 0) {
          if (tau != 0.0) cj[i] = rij;
          if (exact) ref[j] = nj;
          nrm[j] = nj;
        }
      }
    }
    __syncwarp();
    k = i + 1;
  }
  return k;
}

// Householder QR of the first k columns of W without pivoting (the columns
// are already in the wanted order), applied to all w columns: the R factor
// after an exchange of the strong rank-revealing step.
__device__ void warp_qr_fixed(double* W, int h, int w, int k, int lane) {
  for (int i = 0; i < k; ++i) {
    double e, sg;
    pivot_sums(W, h, i, i, e, sg, lane);
    double* ci = W + (size_t)i * h;
    const double alpha = ci[i];
    double tau = 0.0, beta = alpha, sc = 1.0;
    const bool reflect = (sg != 0.0 || alpha < 0.0);
    if (reflect) {
      const double nx = sqrt(alpha * alpha + sg);
      beta = (alpha <= 0.0) ? nx : -nx;
      tau = (beta - alpha) / beta;
      sc = 1.0 / (alpha - beta);
    }
    __syncwarp();
    for (int r = lane; r < h; r += 32) {
      if (r == i) {
        ci[r] = beta;
      } else if (r > i && reflect) {
        ci[r] *= sc;
      }
    }
    __syncwarp();
    if (tau != 0.0) {
      for (int j0 = i + 1; j0 < w; j0 += 4) {
        const int nc = min(4, w - j0);
        double* c0 = W + (size_t)j0 * h;
        double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
        for (int r = i + 1 + lane; r < h; r += 32) {
          const double vr = ci[r];
          d0 = fma(vr, c0[r], d0);
          if (nc > 1) d1 = fma(vr, c0[h + r], d1);
          if (nc > 2) d2 = fma(vr, c0[2 * h + r], d2);
          if (nc > 3) d3 = fma(vr, c0[3 * h + r], d3);
        }
        reduce4(d0, d1, d2, d3, lane);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c >= nc) break;
          double* cj = c0 + (size_t)c * h;
          const double rij = cj[i];
          const double dc = c == 0 ? d0 : c == 1 ? d1 : c == 2 ? d2 : d3;
          const double d = (dc + rij) * tau;
          for (int r = i + 1 + lane; r < h; r += 32) cj[r] = fma(-d, ci[r], cj[r]);
          __syncwarp();
          if (lane == 0) cj[i] = rij - d;
        }
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ long long pad16(long long b) { return (b + 15) & ~15LL; }

__device__ __forceinline__ long long block_record_bytes(int nin, int k) {
  return pad16((long long)sizeof(RecHdr) + pad16(4LL * nin) + 8LL * k * (nin - k));
}

// Reserves one record for the warp; nullptr when the arena is full.
__device__ unsigned char* warp_reserve(const DevBuildArgs& A, long long bytes, int lane) {
  long long off = -1;
  if (lane == 0 && *(volatile int*)A.stop == 0) {
    const unsigned long long o = atomicAdd(A.arena_used, (unsigned long long)bytes);
    if (o + (unsigned long long)bytes <= A.arena_bytes) {
      off = (long long)o;
    } else {
      atomicMin(A.arena_fail, o);
      atomicExch(A.stop, 1);
    }
  }
  off = __shfl_sync(kFull, off, 0);
  return off < 0 ? nullptr : A.arena + off;
}

// Writes the record of one ID block: the skeleton, the redundant columns in
// ascending order and T = R11^{-1} R12 by back substitution, each column of T
// placed at the position of its column in that order.
__device__ void warp_write_block(unsigned char* rec, int unit, int level, int band, int group, int r0, int r1,
                                 int in_off, int nin, int k, const double* W, int h, const int* perm, int lane) {
  if (lane == 0) {
    RecHdr t{};
    t.unit = unit;
    t.kind = 0;
    t.level = level;
    t.band = band;
    t.group = group;
    t.r0 = r0;
    t.r1 = r1;
    t.in_off = in_off;
    t.nin = nin;
    t.k = k;
    t.bytes = block_record_bytes(nin, k);
    *reinterpret_cast<RecHdr*>(rec) = t;
  }
  int* skel = reinterpret_cast<int*>(rec + sizeof(RecHdr));
  int* red = skel + k;
  double* T = reinterpret_cast<double*>(rec + sizeof(RecHdr) + pad16(4LL * nin));
  for (int t = lane; t < k; t += 32) skel[t] = perm[t];
  const int nred = nin - k;
  for (int s = lane; s < nred; s += 32) {
    const int c = perm[k + s];
    int rank = 0;
    for (int s2 = 0; s2 < nred; ++s2) rank += perm[k + s2] < c;
    red[rank] = c;
    const double* rc = W + (size_t)(k + s) * h;
    double* tc = T + (size_t)rank * k;
    for (int t = k - 1; t >= 0; --t) {
      double x = rc[t];
      for (int t2 = t + 1; t2 < k; ++t2) x = fma(-W[(size_t)t2 * h + t], tc[t2], x);
      tc[t] = x / W[(size_t)t * h + t];
    }
  }
}

// Writes the block's record and then runs the strong rank-revealing step of
// Remark QR_algorithm: while some |T(t, s)| > 2, exchange skeleton column t
// with redundant column s, refactor the original columns Z in the new order
// and rewrite the record (at most 2k exchanges; each multiplies |det R11| by
// more than 2).  Returns the number of exchanges.
__device__ int warp_write_strong(unsigned char* rec, int unit, int level, int band, int group, int r0, int r1,
                                 int in_off, int nin, int k, const WarpBuf& B, int h, int lane) {
  int nswap = 0;
  const int nred = nin - k;
  const int* red = reinterpret_cast<const int*>(rec + sizeof(RecHdr)) + k;
  const double* T = reinterpret_cast<const double*>(rec + sizeof(RecHdr) + pad16(4LL * nin));
  for (;;) {
    warp_write_block(rec, unit, level, band, group, r0, r1, in_off, nin, k, B.W, h, B.perm, lane);
    __syncwarp();
    if (k == 0 || nred == 0 || nswap >= 2 * k) break;
    long long best = -1;
    int bi = k * nred;
    for (int x = lane; x < k * nred; x += 32) {
      const long long b = __double_as_longlong(fabs(T[x]));
      if (b > best) {
        best = b;
        bi = x;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const long long ob = __shfl_xor_sync(kFull, best, o);
      const int oi = __shfl_xor_sync(kFull, bi, o);
      if (better(ob, oi, best, bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (!(__longlong_as_double(best) > 2.0)) break;
    // T's column bi / k belongs to redundant column red[bi / k]: find it in perm
    const int c = red[bi / k], t = bi % k;
    int s = -1;
    for (int x = lane; x < nred; x += 32)
      if (B.perm[k + x] == c) s = x;
#pragma unroll
    for (int o = 16; o; o >>= 1) s = max(s, __shfl_xor_sync(kFull, s, o));
    if (s < 0) break;
    __syncwarp();
    if (lane == 0) {
      const int tp = B.perm[t];
      B.perm[t] = B.perm[k + s];
      B.perm[k + s] = tp;
    }
    __syncwarp();
    for (long long x = lane; x < (long long)h * nin; x += 32) {
      const int col = (int)(x / h), i = (int)(x - (long long)col * h);
      B.W[x] = B.Z[(size_t)B.perm[col] * h + i];
    }
    __syncwarp();
    warp_qr_fixed(B.W, h, nin, k, lane);
    ++nswap;
  }
  return nswap;
}

// Marks the unit failed (first reason wins).
__device__ __forceinline__ void set_fail(Shared& S, int why) { atomicCAS(&S.fail, 0, why); }

// Builds unit u; returns its status.
__device__ int build_unit(const DevBuildArgs& A, const Views& V, Shared& S, int u) {
  const int m = u >> 1, p = u & 1, l = A.l, L = 2 * l, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = max(0, (L - m - p + 1) / 2);
  long long* info = A.info + 3LL * u;
  if (n == 0) {
    if (tid == 0) info[0] = info[1] = info[2] = 0;
    return kDone;
  }
  // recurrence coefficients of the n columns, and c_m with
  // P-bar^m_m(x) = c_m (1 - x^2)^{m/2}
  for (int j = tid; j < n; j += kThreads) {
    const int k = m + p + 2 * j;
    V.cinv[j] = 1.0 / rec_c(k, m);
    V.cd[j] = rec_d(k, m);
    V.cm2[j] = j > 0 ? rec_c(k - 2, m) : 0.0;
  }
  if (tid == 0) {
    double cm = 1.0 / sqrt(2.0);
    int ecm = 0;
    for (int j = 1; j <= m; ++j) {
      cm *= sqrt((2.0 * j + 1.0) / (2.0 * j));
      renorm(cm, ecm);
    }
    S.cm = cm;
    S.ecm = ecm;
    S.ngrp = 0;
    S.fail = 0;
    S.swaps = 0;
  }
  __syncthreads();

  // trimming: keep rows up to the last whose weighted norm reaches the
  // threshold.  Only that last row matters, so rows are tried from the pole
  // down, 256 at a time, and each row's sum stops once it reaches the
  // threshold (the sum only grows): the same decision as summing every row.
  int rows = l;
  if (A.trim2 > 0.0) {
    rows = 0;
    for (int top = l; top > 0; top -= kThreads) {
      const int i = top - 1 - tid;
      int last = 0;
      if (i >= 0) {
        double x2, sqw, a, b;
        int e;
        row_init(A, S, m, p, i, x2, sqw, a, b, e);
        double nr = 0.0;
        for (int j = 0; j < n && nr < A.trim2; ++j) {
          const double c = gen_step(V, j, x2, sqw, a, b, e);
          nr = __dadd_rn(nr, __dmul_rn(c, c));
        }
        if (nr >= A.trim2) last = i + 1;
      }
      rows = block_max_int(last, S);
      if (rows > 0) break;
    }
  }
  if (rows == 0) {
    if (tid == 0) info[0] = info[1] = info[2] = 0;
    return kDone;
  }
  const int C = A.C;
  int lam = 0;
  while ((n >> lam) > C) ++lam;
  if (n > C && (n + (1 << lam) - 1) / (1 << lam) > C) ++lam;
  while (lam > 0 && (rows >> lam) < A.min_band_rows) --lam;
  const int nleaves = 1 << lam;
  const int NB = min(kWarps, nleaves);
  if (lam + 1 + NB > kMaxGroups) return kNoScratch;
  for (int g = 0; g < nleaves; ++g) {
    const int wd = (int)((long long)(g + 1) * n / nleaves) - (int)((long long)g * n / nleaves);
    if ((long long)rows * wd > A.buf_words || wd > l) return kNoScratch;
  }

  gen_init(A, V, S, m, p, rows);
  __syncthreads();
  long long sp = 0;
  int ndesc = 0;
  for (int g0 = 0; g0 < nleaves; g0 += NB) {
    // the batch's columns, then its leaf IDs, one per warp
    gen_leaves(A, V, g0, NB, nleaves, n, rows);
    __syncthreads();
    if (warp < NB) {
      const int g = g0 + warp;
      const int c0 = (int)((long long)g * n / nleaves), wd = (int)((long long)(g + 1) * n / nleaves) - c0;
      const WarpBuf B = warp_buf(A, V, warp);
      for (long long t = lane; t < (long long)rows * wd; t += 32) B.W[t] = B.Z[t];
      __syncwarp();
      const int k = warp_cpqr(B.W, rows, wd, A.eps2, B, lane);
      unsigned char* rec = warp_reserve(A, block_record_bytes(wd, k), lane);
      if (rec) {
        const int sw = warp_write_strong(rec, u, 1, 0, g, 0, rows, c0, wd, k, B, rows, lane);
        if (lane == 0 && sw) atomicAdd(&S.swaps, sw);
      } else if (lane == 0) {
        set_fail(S, kNoArena);
      }
      if (lane == 0) S.kres[warp] = k;
    }
    __syncthreads();
    if (S.fail) return S.fail;
    // push the leaves in order: their skeleton columns go on the stack
    for (int q = 0; q < NB; ++q) {
      const int k = S.kres[q];
      if (sp + (long long)rows * k > A.stack_words || ndesc + 1 > A.desc_cap) return kNoScratch;
      const WarpBuf B = warp_buf(A, V, q);
      for (long long t = tid; t < (long long)rows * k; t += kThreads) {
        const int c = (int)(t / rows), i = (int)(t - (long long)c * rows);
        V.stack[sp + t] = B.Z[(size_t)B.perm[c] * rows + i];
      }
      if (tid == 0) {
        V.desc[ndesc] = BandDesc{0, rows, k, 0, sp};
        S.grp[S.ngrp] = GroupDesc{1, g0 + q, 1, ndesc};
        S.ngrp += 1;
      }
      sp += (long long)rows * k;
      ndesc += 1;
    }
    __syncthreads();

    // merge rounds: all pairs of same-level groups at the top of the stack
    for (;;) {
      const int ng = S.ngrp;
      if (ng < 2) break;
      const int lev = S.grp[ng - 1].level;
      int run = 1;
      while (run < ng && S.grp[ng - 1 - run].level == lev) ++run;
      const int P = run / 2;
      if (P == 0) break;
      const int gb = ng - 2 * P;
      const int nb = S.grp[gb].nb;
      const int T = P * 2 * nb;  // ID blocks of this round, two per band of each pair
      for (int q = 0; q < P; ++q) {
        const GroupDesc Lg = S.grp[gb + 2 * q], Rg = S.grp[gb + 2 * q + 1];
        if ((Lg.g & 1) || Rg.g != Lg.g + 1 || Lg.nb != nb || Rg.nb != nb) return kNoScratch;
      }
      if (ndesc + T > A.desc_cap) return kNoScratch;
      const long long base = sp;
      if (tid == 0) S.tmp_sp = (unsigned long long)base;
      __syncthreads();
      for (int t = warp; t < T; t += kWarps) {
        const int q = t / (2 * nb), beta = (t - q * 2 * nb) >> 1, half = t & 1;
        const GroupDesc Lg = S.grp[gb + 2 * q], Rg = S.grp[gb + 2 * q + 1];
        const BandDesc BL = V.desc[Lg.d0 + beta], BR = V.desc[Rg.d0 + beta];
        const int h = BL.r1 - BL.r0, mid = BL.r0 + h / 2, kin = BL.k + BR.k;
        const int rr0 = half ? mid : BL.r0, rr1 = half ? BL.r1 : mid, hh = rr1 - rr0;
        if ((long long)hh * kin > A.buf_words || kin > l) {
          if (lane == 0) set_fail(S, kNoScratch);
          continue;
        }
        const WarpBuf B = warp_buf(A, V, warp);
        // Z = [rows rr0..rr1 of the left band's skeleton columns, then the right's]
        for (long long x = lane; x < (long long)hh * kin; x += 32) {
          const int c = (int)(x / hh), i = (int)(x - (long long)c * hh);
          const double z = c < BL.k ? V.stack[BL.off + (long long)c * h + (rr0 - BL.r0) + i]
                                    : V.stack[BR.off + (long long)(c - BL.k) * h + (rr0 - BL.r0) + i];
          B.Z[x] = z;
          B.W[x] = z;
        }
        __syncwarp();
        const int k = warp_cpqr(B.W, hh, kin, A.eps2, B, lane);
        unsigned char* rec = warp_reserve(A, block_record_bytes(kin, k), lane);
        if (!rec) {
          if (lane == 0) set_fail(S, kNoArena);
          continue;
        }
        const int sw = warp_write_strong(rec, u, lev + 1, 2 * beta + half, Lg.g / 2, rr0, rr1, 0, kin, k, B, hh, lane);
        if (lane == 0 && sw) atomicAdd(&S.swaps, sw);
        // the new band's skeleton columns go to temporary space above the stack
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(&S.tmp_sp, (unsigned long long)hh * k);
        off = __shfl_sync(kFull, off, 0);
        if ((long long)off + (long long)hh * k > A.stack_words) {
          if (lane == 0) set_fail(S, kNoScratch);
          continue;
        }
        for (long long x = lane; x < (long long)hh * k; x += 32) {
          const int c = (int)(x / hh), i = (int)(x - (long long)c * hh);
          V.stack[off + x] = B.Z[(size_t)B.perm[c] * hh + i];
        }
        if (lane == 0) V.desc[ndesc + t] = BandDesc{rr0, rr1, k, 0, (long long)off};
      }
      __syncthreads();
      if (S.fail) return S.fail;
      // the new groups replace the merged ones: final offsets in band order
      // (their words never exceed the merged groups', so every destination
      // lies below `base` and every source above it)
      const int d_run = S.grp[gb].d0;
      if (tid == 0) {
        long long o = V.desc[d_run].off;
        for (int t = 0; t < T; ++t) {
          BandDesc d = V.desc[ndesc + t];
          const long long words = (long long)(d.r1 - d.r0) * d.k;
          d.off = o;
          V.desc[d_run + t] = d;
          o += words;
        }
        S.new_sp = o;
        for (int q = 0; q < P; ++q) {
          const GroupDesc Lg = S.grp[gb + 2 * q];
          S.grp[gb + q] = GroupDesc{lev + 1, Lg.g / 2, 2 * nb, d_run + q * 2 * nb};
        }
        S.ngrp = gb + P;
        if (o > base) S.fail = kNoScratch;
      }
      __syncthreads();
      if (S.fail) return S.fail;
      for (int t = warp; t < T; t += kWarps) {
        const BandDesc src = V.desc[ndesc + t], dst = V.desc[d_run + t];
        const long long words = (long long)(src.r1 - src.r0) * src.k;
        for (long long x = lane; x < words; x += 32) V.stack[dst.off + x] = V.stack[src.off + x];
      }
      sp = S.new_sp;
      ndesc = d_run + T;
      __syncthreads();
    }
  }
  if (S.ngrp != 1) return kNoScratch;
  // the top level's bands: their stored skeleton columns are the final blocks
  const GroupDesc top = S.grp[0];
  for (int beta = warp; beta < top.nb; beta += kWarps) {
    const BandDesc B = V.desc[top.d0 + beta];
    const long long words = (long long)(B.r1 - B.r0) * B.k;
    const long long bytes = pad16((long long)sizeof(RecHdr) + 8 * words);
    unsigned char* rec = warp_reserve(A, bytes, lane);
    if (!rec) {
      if (lane == 0) set_fail(S, kNoArena);
      continue;
    }
    if (lane == 0) {
      RecHdr t{};
      t.unit = u;
      t.kind = 1;
      t.band = beta;
      t.r0 = B.r0;
      t.r1 = B.r1;
      t.k = B.k;
      t.bytes = bytes;
      *reinterpret_cast<RecHdr*>(rec) = t;
    }
    double* Sv = reinterpret_cast<double*>(rec + sizeof(RecHdr));
    for (long long x = lane; x < words; x += 32) Sv[x] = V.stack[B.off + x];
  }
  __syncthreads();
  if (S.fail) return S.fail;
  if (tid == 0) {
    info[0] = rows;
    info[1] = lam;
    info[2] = S.swaps;
  }
  return kDone;
}

__global__ void __launch_bounds__(kThreads, 4) factor_units_kernel(DevBuildArgs A) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Shared S;
  const int l = A.l;
  Views V;
  V.cinv = reinterpret_cast<double*>(dyn);
  V.cd = V.cinv + l;
  V.cm2 = V.cd + l;
  double* g = A.scratch + (long long)blockIdx.x * A.scratch_words;
  V.x2 = g;
  V.sqw = g + l;
  V.ga = g + 2 * l;
  V.gb = g + 3 * l;
  V.ge = reinterpret_cast<int*>(g + 4 * l);
  V.desc = reinterpret_cast<BandDesc*>(g + 5 * l);
  V.warps = g + 5 * l + 3 * A.desc_cap;
  V.warp_words = A.warp_words;
  V.stack = V.warps + kWarps * A.warp_words;
  for (;;) {
    if (threadIdx.x == 0) S.q = (*(volatile int*)A.stop) ? A.n_queue : (int)atomicAdd(A.next, 1u);
    __syncthreads();
    const int q = S.q;
    __syncthreads();
    if (q >= A.n_queue) break;
    const int u = A.queue[q];
    const int st = build_unit(A, V, S, u);
    __syncthreads();
    if (threadIdx.x == 0) A.status[u] = st;
  }
}

size_t dyn_smem(int l) { return (size_t)l * 3 * sizeof(double); }

int leaf_levels(int n, int rows, int C, int mbr) {
  int lam = 0;
  while ((n >> lam) > C) ++lam;
  if (n > C && (n + (1 << lam) - 1) / (1 << lam) > C) ++lam;
  while (lam > 0 && (rows >> lam) < mbr) --lam;
  return lam;
}

struct CudaBuf {
  void* p = nullptr;
  ~CudaBuf() { cudaFree(p); }
};

void check(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    throw std::bad_alloc();  // reported as SHT_ERR_OOM
  }
  if (e != cudaSuccess) throw DeviceError(std::string("device build: ") + what + ": " + cudaGetErrorString(e));
}

}  // namespace

void build_factorizations_device(PlanHost& P, bool fp32, int device) {
  const int l = P.l, L = 2 * l, C = P.leaf_cols, mbr = P.min_band_rows;
  const double eps = fp32 ? P.eps_fp32 : P.eps_id;
  std::vector<UnitFact>& out = fp32 ? P.fact32 : P.fact64;
  out.assign((size_t)L * 2, UnitFact());
  check(cudaSetDevice(device), "cudaSetDevice");

  // Scratch bounds per CTA, over every unit and every number of kept rows:
  // a leaf or merge block holds at most (rows + 2^lam) x (leaf width)
  // values; a group at level j at most rows x min(rows / 2^(j-1) + 1,
  // 2^(j-1) x leaf width).  The stack holds one group per level, a batch of
  // up to kBatch leaves, and the new groups of a merge round before they
  // move down.
  long long buf_words = 1, stack_words = 1;
  int max_lam = 0;
  for (int n = 1; n <= l; ++n) {
    const int lam0 = leaf_levels(n, l, C, 0);
    for (int lam = 0; lam <= lam0; ++lam) {
      // the most rows for which the band rule leaves lam levels
      long long rows = l;
      if (lam < lam0 && mbr > 0) rows = std::min<long long>(l, (long long)mbr << (lam + 1));
      const long long wd = (n + (1LL << lam) - 1) >> lam;
      buf_words = std::max(buf_words, (rows + (1LL << lam)) * wd);
      long long sum = 0, gmax = 0;
      for (int j = 1; j <= lam + 1; ++j) {
        const long long gj = rows * std::min(((rows + (1LL << (j - 1)) - 1) >> (j - 1)) + 1, (1LL << (j - 1)) * wd);
        sum += gj;
        gmax = std::max(gmax, gj);
      }
      const long long batch = (long long)std::min(kBatch, 1 << lam) * rows * std::min(rows + 1, wd);
      stack_words = std::max(stack_words, sum + gmax + 2 * batch);
      max_lam = std::max(max_lam, lam);
    }
  }
  const long long desc_cap = (4LL << (max_lam + 1)) + 4 * kBatch;
  // per warp: Z and W (buf_words each), nrm and ref (l each), perm (l ints)
  const long long warp_words = 2 * buf_words + 3LL * l;
  const long long scratch_words = 5LL * l + 3 * desc_cap + kWarps * warp_words + stack_words;

  int sms = 0;
  check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device), "SM count");
  const size_t smem = dyn_smem(l);
  check(cudaFuncSetAttribute(factor_units_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "shared memory limit");
  int per_sm = 0;
  check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_units_kernel, kThreads, smem), "occupancy");
  per_sm = std::max(1, std::min(per_sm, 4));
  size_t free_b = 0, total_b = 0;
  check(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
  long long ctas = std::min<long long>((long long)sms * per_sm, 2LL * L);
  // scratch at most a quarter of the free memory
  ctas = std::min<long long>(ctas, (long long)(free_b / 4 / (8 * (size_t)scratch_words)));
  if (ctas < 1) throw std::runtime_error("device build: not enough device memory for one CTA's scratch");
  // arena: half the dense operator (the butterflies store about a third of
  // it at eps_id = 1e-12), at most a quarter of the free memory
  long long dense = 0;
  for (int m = 0; m < L; ++m)
    for (int p = 0; p < 2; ++p) dense += (long long)l * std::max(0, (L - m - p + 1) / 2);
  unsigned long long arena_bytes =
      std::min<unsigned long long>(4ULL * dense + (64ULL << 20), free_b / 4);
  if (P.device_arena_bytes > 0) arena_bytes = std::min<unsigned long long>(arena_bytes, P.device_arena_bytes);
  arena_bytes &= ~15ULL;

  // node data, as the host's column generator computes it
  std::vector<double> xpos(l), spos(l), sq2w(l);
  for (int i = 0; i < l; ++i) {
    xpos[i] = P.x[l + i];
    spos[i] = P.sin_pos[i];
    sq2w[i] = std::sqrt(2.0 * P.w[l + i]);
  }
  std::vector<int> order(2 * L);
  for (int u = 0; u < 2 * L; ++u) order[u] = u;
  std::stable_sort(order.begin(), order.end(), [](int a, int b) { return (a / 2) < (b / 2); });

  CudaBuf d_nodes, d_queue, d_ctl, d_status, d_info, d_scratch, d_arena;
  check(cudaMalloc(&d_nodes.p, 3 * sizeof(double) * l), "cudaMalloc nodes");
  check(cudaMalloc(&d_queue.p, sizeof(int) * 2 * L), "cudaMalloc queue");
  check(cudaMalloc(&d_ctl.p, 64), "cudaMalloc control");
  check(cudaMalloc(&d_status.p, sizeof(int) * 2 * L), "cudaMalloc status");
  check(cudaMalloc(&d_info.p, sizeof(long long) * 3 * 2 * L), "cudaMalloc info");
  check(cudaMalloc(&d_scratch.p, 8 * (size_t)scratch_words * ctas), "cudaMalloc scratch");
  check(cudaMalloc(&d_arena.p, arena_bytes), "cudaMalloc arena");
  double* dn = static_cast<double*>(d_nodes.p);
  check(cudaMemcpy(dn, xpos.data(), 8 * l, cudaMemcpyHostToDevice), "copy nodes");
  check(cudaMemcpy(dn + l, spos.data(), 8 * l, cudaMemcpyHostToDevice), "copy nodes");
  check(cudaMemcpy(dn + 2 * l, sq2w.data(), 8 * l, cudaMemcpyHostToDevice), "copy nodes");
  check(cudaMemset(d_status.p, 0, sizeof(int) * 2 * L), "clear status");

  DevBuildArgs A{};
  A.l = l;
  A.C = C;
  A.min_band_rows = mbr;
  A.eps2 = eps * eps;
  const double thr = P.trim_eps > 0.0 ? P.trim_eps / std::sqrt((double)l) : 0.0;
  A.trim2 = thr * thr;
  A.xpos = dn;
  A.spos = dn + l;
  A.sq2w = dn + 2 * l;
  A.queue = static_cast<int*>(d_queue.p);
  unsigned char* ctl = static_cast<unsigned char*>(d_ctl.p);
  A.next = reinterpret_cast<unsigned*>(ctl);
  A.stop = reinterpret_cast<int*>(ctl + 4);
  A.arena_used = reinterpret_cast<unsigned long long*>(ctl + 8);
  A.arena_fail = reinterpret_cast<unsigned long long*>(ctl + 16);
  A.scratch = static_cast<double*>(d_scratch.p);
  A.scratch_words = scratch_words;
  A.buf_words = buf_words;
  A.stack_words = stack_words;
  A.desc_cap = desc_cap;
  A.warp_words = warp_words;
  A.arena = static_cast<unsigned char*>(d_arena.p);
  A.arena_bytes = arena_bytes;
  A.status = static_cast<int*>(d_status.p);
  A.info = static_cast<long long*>(d_info.p);

  std::vector<int> status(2 * L, kPending);
  std::vector<long long> info(3 * 2 * L);
  ByteBuf host;
  std::vector<int> pending = order;
  // CTAs per launch: all of them, or one when a launch finished no block
  // (its blocks' records crowded each other out of the arena)
  long long grid_limit = ctas;
  while (!pending.empty()) {
    check(cudaMemcpy(d_queue.p, pending.data(), sizeof(int) * pending.size(), cudaMemcpyHostToDevice), "queue");
    struct {
      unsigned next;
      int stop;
      unsigned long long used, fail;
    } c0{0, 0, 0, ~0ULL};
    check(cudaMemcpy(ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice), "control");
    A.n_queue = (int)pending.size();
    const int grid = (int)std::min<long long>(grid_limit, (long long)pending.size());
    const auto t0 = std::chrono::steady_clock::now();
    factor_units_kernel<<<grid, kThreads, smem>>>(A);
    check(cudaGetLastError(), "launch");
    check(cudaDeviceSynchronize(), "factor_units_kernel");
    P.t_factor_kernel += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    check(cudaMemcpy(status.data(), d_status.p, sizeof(int) * 2 * L, cudaMemcpyDeviceToHost), "status");
    check(cudaMemcpy(info.data(), d_info.p, sizeof(long long) * 3 * 2 * L, cudaMemcpyDeviceToHost), "info");
    check(cudaMemcpy(&c0, ctl, sizeof(c0), cudaMemcpyDeviceToHost), "control");
    for (int u : pending)
      if (status[u] == kNoScratch)
        throw std::runtime_error("device build: unit " + std::to_string(u) + " exceeded its scratch bound");
    const unsigned long long limit = std::min(c0.used, std::min(c0.fail, arena_bytes));
    host.resize(limit);
    if (limit) check(cudaMemcpy(host.data(), d_arena.p, limit, cudaMemcpyDeviceToHost), "arena");

    // records of the units finished in this wave, in emission order
    std::vector<std::vector<size_t>> recs(2 * L);
    for (unsigned long long off = 0; off + sizeof(RecHdr) <= limit;) {
      RecHdr h;
      std::memcpy(&h, host.data() + off, sizeof h);
      if (h.bytes < (long long)sizeof(RecHdr) || off + (unsigned long long)h.bytes > limit || h.unit < 0 ||
          h.unit >= 2 * L)
        throw std::runtime_error("device build: corrupt record at offset " + std::to_string(off));
      if (status[h.unit] == kDone) recs[h.unit].push_back(off);
      off += (unsigned long long)h.bytes;
    }
    std::vector<int> done, next_wave;
    for (int u : pending) (status[u] == kDone ? done : next_wave).push_back(u);
    if (done.empty()) {
      if (grid_limit == 1) throw std::invalid_argument("device build: the output arena cannot hold one unit");
      grid_limit = 1;
      continue;
    }

    std::atomic<int> cursor(0);
    int nt = P.num_threads > 0 ? P.num_threads : (int)std::thread::hardware_concurrency();
    nt = std::max(1, std::min(nt, 256));
    std::vector<std::string> errors(nt);
    auto worker = [&](int tid) {
      try {
        for (;;) {
          const int q = cursor.fetch_add(1);
          if (q >= (int)done.size()) break;
          const int u = done[q];
          UnitFact U;
          U.m = u / 2;
          U.p = u % 2;
          U.n = std::max(0, (L - U.m - U.p + 1) / 2);
          U.rows = (int)info[3 * u];
          U.levels = (int)info[3 * u + 1];
          U.swaps = info[3 * u + 2];
          std::vector<FinalBlock> top;
          for (size_t off : recs[u]) {
            RecHdr h;
            std::memcpy(&h, host.data() + off, sizeof h);
            const unsigned char* body = host.data() + off + sizeof(RecHdr);
            if (h.kind == 0) {
              IdBlock b;
              b.level = h.level;
              b.band = h.band;
              b.group = h.group;
              b.r0 = h.r0;
              b.r1 = h.r1;
              b.in_off = h.in_off;
              b.nin = h.nin;
              b.k = h.k;
              const int* ix = reinterpret_cast<const int*>(body);
              b.skel.assign(ix, ix + h.k);
              b.red.assign(ix + h.k, ix + h.nin);
              b.T.resize((size_t)h.k * (h.nin - h.k));
              std::memcpy(b.T.data(), body + ((4LL * h.nin + 15) & ~15LL), 8 * b.T.size());
              U.blocks.push_back(std::move(b));
            } else {
              FinalBlock f;
              f.band = h.band;
              f.r0 = h.r0;
              f.r1 = h.r1;
              f.k = h.k;
              f.S.resize((size_t)(h.r1 - h.r0) * h.k);
              std::memcpy(f.S.data(), body, 8 * f.S.size());
              top.push_back(std::move(f));
            }
          }
          if (U.n > 0 && U.rows > 0) {
            // records arrive in whatever order the warps finished: put the
            // blocks in the host's depth-first creation order (a group is
            // made right after the last leaf under it; lower levels first)
            // and the top bands in band order, so that the streams do not
            // depend on timing
            auto created = [](const IdBlock& b) {
              return std::make_tuple(((long long)b.group + 1) << (b.level - 1), b.level, b.band);
            };
            std::sort(U.blocks.begin(), U.blocks.end(),
                      [&](const IdBlock& x, const IdBlock& y) { return created(x) < created(y); });
            std::sort(top.begin(), top.end(), [](const FinalBlock& x, const FinalBlock& y) { return x.band < y.band; });
            // the host's depth-first order, replayed from the ranks: its
            // peak memory (the device batches leaves, so its own differs)
            U.peak_words = depth_first_peak(U);
            finish_unit(P, U, std::move(top));
          }
          out[u] = std::move(U);
        }
      } catch (const std::exception& e) {
        errors[tid] = e.what();
        cursor.store((int)done.size());
      }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(worker, t);
    worker(0);
    for (auto& t : th) t.join();
    for (auto& e : errors)
      if (!e.empty()) throw std::runtime_error(e);
    pending.swap(next_wave);
  }
}

}  // namespace sht
