// phi.cu -- half-sample phase of the phi stage (Section 2, eq. phis).
//
// With phi_j = 2 pi (j + 1/2)/N, N = 4l - 1, the sums over m of eq.
// alternate_expansion become an FFT of length N once G^m is multiplied by
// e^{i pi m / N} (synthesis); the analysis multiplies the FFT output by
// e^{-i pi m / N} / N.  These kernels apply that per-order phase to a
// [2l][2l] complex array; the full transforms fuse it into the sweep instead.
#include <cuda_runtime.h>

#include "kernels.h"

namespace sht {
namespace {

template <class T>
struct Cplx;
template <>
struct Cplx<double> {
  using type = double2;
};
template <>
struct Cplx<float> {
  using type = float2;
};

template <class T>
__global__ void phase_kernel(const typename Cplx<T>::type* __restrict__ src, typename Cplx<T>::type* dst,
                             const double2* __restrict__ tw, int L) {
  const size_t n = (size_t)L * L;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(e / L);
    const double2 t = tw[m];
    const auto g = src[e];
    const double re = (double)g.x * t.x - (double)g.y * t.y;
    const double im = (double)g.x * t.y + (double)g.y * t.x;
    dst[e].x = (T)re;
    dst[e].y = (T)im;
  }
}

}  // namespace

cudaError_t phase_launch(bool fp32, const void* src, void* dst, const double2* tw, int l, int num_sms,
                         cudaStream_t st) {
  const int L = 2 * l;
  const size_t n = (size_t)L * L;
  const int block = 256;
  const int grid = (int)std::min<size_t>((n + block - 1) / block, (size_t)num_sms * 8);
  if (fp32)
    phase_kernel<float><<<grid, block, 0, st>>>(reinterpret_cast<const float2*>(src), reinterpret_cast<float2*>(dst),
                                                tw, L);
  else
    phase_kernel<double><<<grid, block, 0, st>>>(reinterpret_cast<const double2*>(src),
                                                 reinterpret_cast<double2*>(dst), tw, L);
  return cudaGetLastError();
}

}  // namespace sht
