// direct.cu -- direct float64 Legendre stage (the O(l^3) method of Section 2)
// with the dense operator stored in HBM.  Baseline for the butterfly.
//
// Storage: for each order m and parity p, the block P-bar^m_{m+p+2j}(x_{l+i})
// (j < n_{m,p}, i < rows_{m,p}) in [j][i] layout, i fastest.
//   synthesis: one CTA per (m, tile of 128 node rows); thread i forms
//              E_i = sum_j P_even[j][i] beta_even[j] and O_i likewise (coalesced
//              loads down the columns), then unfolds G(x_{l+i}) = E + O,
//              G(x_{l-1-i}) = E - O (Section 2.3 parity).
//   analysis:  one CTA per (m, p); folds u_i = w_i (G(x_{l+i}) +- G(x_{l-1-i}))
//              into shared memory, then each warp forms beta_j = sum_i P[j][i] u_i
//              with lanes along i and a shuffle reduction.
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

__global__ void __launch_bounds__(256) direct_analysis_kernel(const DirectArgs A) {
  extern __shared__ double2 us[];  // [rows]
  const int l = A.l, L = 2 * l;
  const int m = blockIdx.x, p = blockIdx.y;
  const int u = 2 * m + p;
  const int n = A.ncol[u], rows = A.rows[u];
  if (n == 0) return;
  const double2* G = reinterpret_cast<const double2*>(A.in) + (size_t)m * L;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    const double2 gp = G[l + i], gm = G[l - 1 - i];
    const double w = A.w_pos[i];
    us[i] = p == 0 ? make_double2(w * (gp.x + gm.x), w * (gp.y + gm.y))
                   : make_double2(w * (gp.x - gm.x), w * (gp.y - gm.y));
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* beta = reinterpret_cast<double2*>(A.out) + tri_off(m, L) + p;
  for (int j = warp; j < n; j += 8) {
    const double* D = A.dense + A.off[u] + (size_t)j * rows;
    double ar = 0, ai = 0;
    for (int i = lane; i < rows; i += 32) {
      const double a = D[i];
      ar = fma(a, us[i].x, ar);
      ai = fma(a, us[i].y, ai);
    }
    for (int o = 16; o; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) beta[2 * (size_t)j] = make_double2(ar, ai);
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
  const dim3 grid(2 * l, 2);
  const size_t smem = sizeof(double2) * (size_t)l;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(direct_analysis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(double2) * 1024);
    if (e != cudaSuccess) return e;
  }
  direct_analysis_kernel<<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sht
