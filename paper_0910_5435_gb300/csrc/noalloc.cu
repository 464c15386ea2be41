// noalloc.cu -- a Legendre synthesis entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc on their compute path: a real-time
// loop that may not block on the device-wide synchronization an allocation
// can cause, an application whose memory pools own the whole device, or a
// host framework that forbids allocation between its set-up and tear-down
// phases.  sht_legendre_synthesize (capi.cu) allocates nothing once its
// precision is on the device, but it may build and upload a precision on
// first use, and its work-queue counter and status word live in memory the
// plan allocated.  This entry point never builds or uploads anything.  It
// takes the sweep kernel's scratch (the counter and the status word) from a
// file-scope device array, located once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/sht.h"
#include "kernels.h"
#include "plan_access.h"

namespace {

// One slot per independent launch: word 0 = work-queue counter, word 1 =
// status word; padded to 32 bytes so that slots share no sector.
constexpr int kSlotWords = 8;
static __device__ __align__(256) unsigned g_sweep_scratch[SHT_NOALLOC_MAX_SLOTS * kSlotWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned* g_scratch_ptr[kMaxDevices] = {};

// Set-up for `device` (already current): the array's address on that
// device, looked up once.  The array is zero at module load; every call
// clears its slot again in stream order before the launch.
sht_status scratch_for(int device, unsigned** out) {
  if (device < 0 || device >= kMaxDevices) return SHT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_ptr[device]) {
    unsigned* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_sweep_scratch);
    if (e != cudaSuccess) {
      sht::set_error_detail("cudaGetSymbolAddress", cudaGetErrorString(e));
      return SHT_ERR_CUDA;
    }
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return SHT_OK;
}

// Restores the caller's current device when the entry point returns.
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" sht_status sht_legendre_synthesize_noalloc(sht_plan_t plan, sht_precision prec, const void* beta,
                                                      void* G, int slot, unsigned* status,
                                                      sht_stream_t stream) {
  if (slot < 0 || slot >= SHT_NOALLOC_MAX_SLOTS) {
    char what[96];
    snprintf(what, sizeof(what), "slot %d is outside the %d static scratch slots", slot, SHT_NOALLOC_MAX_SLOTS);
    sht::set_error_detail("sht_legendre_synthesize_noalloc", what);
    return SHT_ERR_INVALID_ARG;
  }
  if (status && (reinterpret_cast<uintptr_t>(status) % alignof(unsigned)) != 0) {
    sht::set_error_detail("sht_legendre_synthesize_noalloc", "status word is not 4-byte aligned");
    return SHT_ERR_INVALID_ARG;
  }
  sht::PreparedSweep L;
  sht_status s = sht::prepared_sweep(plan, prec, 0, beta, G, &L);
  if (s != SHT_OK) return s;
  DeviceGuard keep;  // the plan's device is made current; the caller's comes back on return
  cudaError_t e = cudaSetDevice(L.device);
  if (e != cudaSuccess) {
    sht::set_error_detail("cudaSetDevice", cudaGetErrorString(e));
    return SHT_ERR_CUDA;
  }
  unsigned* base = nullptr;
  s = scratch_for(L.device, &base);
  if (s != SHT_OK) return s;
  unsigned* word = base + (size_t)slot * kSlotWords;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the counter and the status word must start at zero; a launch that gave up
  // early leaves its counter dirty, so they are cleared in stream order
  L.args.counter = word;
  L.args.status = status ? status : word + 1;
  if ((e = cudaMemsetAsync(word, 0, 2 * sizeof(unsigned), st)) != cudaSuccess ||
      (status && (e = cudaMemsetAsync(status, 0, sizeof(unsigned), st)) != cudaSuccess)) {
    sht::set_error_detail("cudaMemsetAsync", cudaGetErrorString(e));
    return SHT_ERR_CUDA;
  }
  // the launch's own result; an error the caller left pending on this thread
  // is neither cleared nor reported here
  if ((e = sht::sweep_launch(L.prec, L.consumer_warps, L.args, L.grid, L.smem, st)) != cudaSuccess) {
    sht::set_error_detail("sweep launch", cudaGetErrorString(e));
    return SHT_ERR_CUDA;
  }
  return SHT_OK;
}
