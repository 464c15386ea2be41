// peak.cu -- float64 FMA throughput of the device: the ceiling the float64
// kernels are compared with, measured rather than assumed; and the float64
// tensor-core (warp MMA) throughput beside it, which decides whether block
// products over several right-hand sides could gain from tensor cores.
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

// The same for the float64 tensor-core product: every warp runs kMmaChains
// independent accumulations D <- A B + D of the 8x8x4 float64 warp MMA
// (256 FMAs per instruction), operands in registers.
constexpr int kMmaChains = 8;

__global__ void __launch_bounds__(kThreads) dmma_loop_kernel(double* sink, int iters, double a, double b) {
  double d[kMmaChains][2];
#pragma unroll
  for (int c = 0; c < kMmaChains; ++c) {
    d[c][0] = 1e-3 * (threadIdx.x + c);
    d[c][1] = 1e-3 * (threadIdx.x + 2 * c);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kMmaChains; ++c)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
          : "+d"(d[c][0]), "+d"(d[c][1])
          : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kMmaChains; ++c) s += d[c][0] + d[c][1];
  if (s == -1.0) sink[blockIdx.x] = s;
}

// Times one launch of `launch(iters)` with CUDA events (after a warm-up
// launch of the same size), growing iters by 4x from iters0 until a launch
// lasts over 40 ms (at most six sizes); returns the iterations and the
// milliseconds of the last timed launch.
template <class Launch>
sht_status time_loop(int iters0, Launch launch, int* iters_out, float* ms_out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sht_status st = SHT_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = SHT_ERR_CUDA;
  int iters = iters0;
  float ms = 0.f;
  for (int rep = 0; st == SHT_OK && rep < 6; ++rep) {
    launch(iters);
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = SHT_ERR_CUDA;
      break;
    }
    if (ms > 40.f) break;
    if (rep + 1 < 6) iters *= 4;
  }
  if (st == SHT_OK && cudaGetLastError() != cudaSuccess) st = SHT_ERR_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *iters_out = iters;
  *ms_out = ms;
  return st;
}

sht_status sm_count(int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SHT_ERR_CUDA;
  if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SHT_ERR_CUDA;
  return SHT_OK;
}

}  // namespace

extern "C" sht_status sht_measure_fp64_mma(double* tflops) {
  if (!tflops) return SHT_ERR_INVALID_ARG;
  *tflops = 0.0;
  int sms = 0;
  sht_status st = sm_count(&sms);
  if (st != SHT_OK) return st;
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * 8 * sms) != cudaSuccess) return SHT_ERR_OOM;
  const int blocks = 8 * sms;  // 2048 threads per SM
  const double a = 1e-3, b = 1e-3;
  int iters = 0;
  float ms = 0.f;
  st = time_loop(1 << 9, [&](int it) { dmma_loop_kernel<<<blocks, kThreads>>>(sink, it, a, b); }, &iters, &ms);
  // 8 x 8 x 4 FMAs per warp instruction, 2 flops each
  if (st == SHT_OK && ms > 0.f)
    *tflops = 2.0 * 256.0 * kMmaChains * (double)iters * blocks * (kThreads / 32) / (ms * 1e-3) / 1e12;
  cudaFree(sink);
  return st;
}

extern "C" sht_status sht_measure_fp64_fma(double* tflops) {
  if (!tflops) return SHT_ERR_INVALID_ARG;
  *tflops = 0.0;
  int sms = 0;
  sht_status st = sm_count(&sms);
  if (st != SHT_OK) return st;
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * 8 * sms) != cudaSuccess) return SHT_ERR_OOM;
  const int blocks = 8 * sms;  // 2048 threads per SM
  const double a = 1.0 - 1e-12, b = 1e-9;
  int iters = 0;
  float ms = 0.f;
  st = time_loop(1 << 12, [&](int it) { fma_loop_kernel<<<blocks, kThreads>>>(sink, it, a, b); }, &iters, &ms);
  if (st == SHT_OK && ms > 0.f)
    *tflops = 2.0 * kChains * (double)iters * blocks * kThreads / (ms * 1e-3) / 1e12;
  cudaFree(sink);
  return st;
}
