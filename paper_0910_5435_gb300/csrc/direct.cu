// direct.cu -- direct float64 Legendre stage (the O(l^3) method of Section 2)
// with the dense operator stored in HBM.  Baseline for the butterfly.
//
// Storage: for each order m and parity p, the block P-bar^m_{m+p+2j}(x_{l+i})
// (j < n_{m,p}, i < rows_{m,p}) in [j][i] layout, i fastest.
//   synthesis: one CTA per (m, tile of 128 node rows); thread i forms
//              E_i = sum_j P_even[j][i] beta_even[j] and O_i likewise (coalesced
//              loads down the columns), then unfolds G(x_{l+i}) = E + O,
//              G(x_{l-1-i}) = E - O (Section 2.3 parity).
//   analysis:  one CTA per (m, p, tile of 128 columns j); folds
//              u_i = w_i (G(x_{l+i}) +- G(x_{l-1-i})) into shared memory, then
//              each warp forms beta_j = sum_i P[j][i] u_i for eight columns
//              at once (lanes along i, a transposing shuffle reduction).
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace sht {
namespace {

__device__ __forceinline__ size_t tri_off(int m, int L) { return (size_t)m * L - (size_t)m * (m - 1) / 2; }

constexpr int kRowTile = 128;

__global__ void __launch_bounds__(kRowTile) direct_synth_kernel(const DirectArgs A) {
  extern __shared__ double2 xs[];  // [n0 + n1]
  const int l = A.l, L = 2 * l;
  const int m = blockIdx.y;
  const int u0 = 2 * m, u1 = 2 * m + 1;
  const int n0 = A.ncol[u0], n1 = A.ncol[u1];
  const int r0 = A.rows[u0], r1 = A.rows[u1];
  const double2* beta = reinterpret_cast<const double2*>(A.in) + tri_off(m, L);
  for (int j = threadIdx.x; j < n0; j += blockDim.x) xs[j] = beta[2 * j];
  for (int j = threadIdx.x; j < n1; j += blockDim.x) xs[n0 + j] = beta[2 * j + 1];
  __syncthreads();
  const int i = blockIdx.x * kRowTile + threadIdx.x;
  if (i >= l) return;
  double er = 0, ei = 0, orr = 0, oi = 0;
  if (i < r0) {
    const double* D = A.dense + A.off[u0] + i;
    int j = 0;
    double er1 = 0, ei1 = 0;
    for (; j + 1 < n0; j += 2) {
      const double a = D[(size_t)j * r0], b = D[(size_t)(j + 1) * r0];
      er = fma(a, xs[j].x, er);
      ei = fma(a, xs[j].y, ei);
      er1 = fma(b, xs[j + 1].x, er1);
      ei1 = fma(b, xs[j + 1].y, ei1);
    }
    if (j < n0) {
      const double a = D[(size_t)j * r0];
      er = fma(a, xs[j].x, er);
      ei = fma(a, xs[j].y, ei);
    }
    er += er1;
    ei += ei1;
  }
  if (i < r1) {
    const double* D = A.dense + A.off[u1] + i;
    int j = 0;
    double or1 = 0, oi1 = 0;
    for (; j + 1 < n1; j += 2) {
      const double a = D[(size_t)j * r1], b = D[(size_t)(j + 1) * r1];
      orr = fma(a, xs[n0 + j].x, orr);
      oi = fma(a, xs[n0 + j].y, oi);
      or1 = fma(b, xs[n0 + j + 1].x, or1);
      oi1 = fma(b, xs[n0 + j + 1].y, oi1);
    }
    if (j < n1) {
      const double a = D[(size_t)j * r1];
      orr = fma(a, xs[n0 + j].x, orr);
      oi = fma(a, xs[n0 + j].y, oi);
    }
    orr += or1;
    oi += oi1;
  }
  double2* G = reinterpret_cast<double2*>(A.out) + (size_t)m * L;
  G[l + i] = make_double2(er + orr, ei + oi);
  G[l - 1 - i] = make_double2(er - orr, ei - oi);
}

// Analysis: one CTA per (tile of kColTile columns j, parity p, order m), so
// that the large units of small m spread over many SMs; the grid runs
// m-major (largest units first).  Each CTA folds the unit's node values
// into shared memory (a few percent of the operator's bytes, re-read from L2
// by the unit's other tiles).  Each warp then takes kWarpCols columns at a
// time (two groups per tile), lanes along i: per row it loads kWarpCols coalesced operator values
// and one u_i, and keeps 2 * kWarpCols partial sums.  The lanes' partial
// sums are reduced by a transposing shuffle tree: at each step a lane keeps
// half of its values and adds the partner's copy of that half, so the 16
// sums of 32 lanes take 16 shuffles and 16 additions per lane (2 per column,
// against 10 for a separate reduction of each column), and lane pairs end
// holding one real or imaginary total each.
constexpr int kColTile = 128;
constexpr int kWarpCols = 8;
constexpr int kAnaWarps = 8;  // each takes kColTile / (kAnaWarps * kWarpCols) groups of columns

__global__ void __launch_bounds__(kAnaWarps * 32, 3) direct_analysis_kernel(const DirectArgs A) {
  extern __shared__ double2 us[];  // [rows]
  const int l = A.l, L = 2 * l;
  const int p = blockIdx.y, m = blockIdx.z;
  const int u = 2 * m + p;
  const int n = A.ncol[u], rows = A.rows[u];
  const int j0 = blockIdx.x * kColTile;
  if (j0 >= n) return;
  const double2* G = reinterpret_cast<const double2*>(A.in) + (size_t)m * L;
  const int tid = threadIdx.x;
  for (int i = tid; i < rows; i += kAnaWarps * 32) {
    const double2 gp = G[l + i], gm = G[l - 1 - i];
    const double w = A.w_pos[i];
    us[i] = p == 0 ? make_double2(w * (gp.x + gm.x), w * (gp.y + gm.y))
                   : make_double2(w * (gp.x - gm.x), w * (gp.y - gm.y));
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  for (int jw = j0 + warp * kWarpCols; jw < min(n, j0 + kColTile); jw += kAnaWarps * kWarpCols) {
    const int nc = min(kWarpCols, n - jw);
    const double* D = A.dense + A.off[u] + (size_t)jw * rows;
    double acc[2 * kWarpCols];
#pragma unroll
    for (int v = 0; v < 2 * kWarpCols; ++v) acc[v] = 0.0;
    for (int i = lane; i < rows; i += 32) {
      const double2 x = us[i];
      double a[kWarpCols];
#pragma unroll
      for (int c = 0; c < kWarpCols; ++c) a[c] = c < nc ? D[(size_t)c * rows + i] : 0.0;
#pragma unroll
      for (int c = 0; c < kWarpCols; ++c) {
        acc[2 * c] = fma(a[c], x.x, acc[2 * c]);
        acc[2 * c + 1] = fma(a[c], x.y, acc[2 * c + 1]);
      }
    }
    // transposing reduction: 16 -> 8 -> 4 -> 2 -> 1 values per lane
#pragma unroll
    for (int half = kWarpCols, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
      const bool up = (lane & bit) != 0;  // this lane keeps the upper half
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const double keep = up ? acc[half + k] : acc[k];
        const double give = up ? acc[k] : acc[half + k];
        acc[k] = keep + __shfl_xor_sync(0xffffffffu, give, bit);
      }
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    // lane bits 4..1 name the value: v = 2 c + (0 re, 1 im)
    const int v = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    if ((lane & 1) == 0 && (v >> 1) < nc) {
      double* beta = reinterpret_cast<double*>(reinterpret_cast<double2*>(A.out) + tri_off(m, L) + p);
      beta[2 * 2 * (size_t)(jw + (v >> 1)) + (v & 1)] = acc[0];
    }
  }
}

}  // namespace

cudaError_t direct_synth_launch(const DirectArgs& a, cudaStream_t st) {
  const int l = a.l;
  const dim3 grid((l + kRowTile - 1) / kRowTile, 2 * l);
  const size_t smem = sizeof(double2) * (size_t)(2 * l + 1);
  if (smem > 48 * 1024) {
    // per-kernel setting shared by all plans: never lower it
    cudaError_t e = cudaFuncSetAttribute(direct_synth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(double2) * (2 * 1024 + 1));
    if (e != cudaSuccess) return e;
  }
  direct_synth_kernel<<<grid, kRowTile, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t direct_analysis_launch(const DirectArgs& a, cudaStream_t st) {
  const int l = a.l;
  const dim3 grid((l + kColTile - 1) / kColTile, 2, 2 * l);
  const size_t smem = sizeof(double2) * (size_t)l;
  if (smem > 48 * 1024) {
    // per-kernel setting shared by all plans: set for the largest l
    cudaError_t e = cudaFuncSetAttribute(direct_analysis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(double2) * 1024);
    if (e != cudaSuccess) return e;
  }
  direct_analysis_kernel<<<grid, kAnaWarps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sht
