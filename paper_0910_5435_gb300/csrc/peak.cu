// peak.cu -- float64 FMA throughput of the device: the ceiling the float64
// kernels are compared with, measured rather than assumed.
//
// Every thread runs eight independent chains x <- x * a + b in registers, so
// the loop is bound by the FP64 pipe alone (no memory traffic, enough
// independent work per warp to cover the pipe's latency).

#include <cuda_runtime.h>

#include "../../include/sht.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_loop_kernel(double* sink, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // never true for the arguments used; keeps the loop from being removed
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" sht_status sht_measure_fp64_fma(double* tflops) {
  if (!tflops) return SHT_ERR_INVALID_ARG;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SHT_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SHT_ERR_CUDA;
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * 8 * sms) != cudaSuccess) return SHT_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sht_status st = SHT_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = SHT_ERR_CUDA;
  const int blocks = 8 * sms;  // 2048 threads per SM
  const double a = 1.0 - 1e-12, b = 1e-9;
  int iters = 1 << 12;
  float ms = 0.f;
  for (int rep = 0; st == SHT_OK && rep < 6; ++rep) {
    // grow the loop until one launch lasts about 50 ms, then keep the last
    fma_loop_kernel<<<blocks, kThreads>>>(sink, iters, a, b);
    cudaEventRecord(e0);
    fma_loop_kernel<<<blocks, kThreads>>>(sink, iters, a, b);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = SHT_ERR_CUDA;
      break;
    }
    if (ms > 40.f) break;
    if (rep + 1 < 6) iters *= 4;
  }
  if (st == SHT_OK && cudaGetLastError() != cudaSuccess) st = SHT_ERR_CUDA;
  if (st == SHT_OK && ms > 0.f)
    *tflops = 2.0 * kChains * (double)iters * blocks * kThreads / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}
