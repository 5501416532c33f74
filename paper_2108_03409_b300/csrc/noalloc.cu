// noalloc.cu -- vmc_force_noalloc: the <O> / F reduction of vmc_grad for callers that
// cannot allocate device memory.  Its scratch (energy statistics and the per-chunk FP64
// partial sums) lives in one file-scope device array of fixed size instead of a buffer
// from cudaMalloc, so the entry point itself allocates nothing.
#include <mutex>

#include "vmc.h"
#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

// 2^21 doubles = 16 MiB.  A GPU holds the array from the first call on it (the module is
// placed on a device when it is first used there; with CUDA_MODULE_LOADING=EAGER, from
// library load) until the process exits.
static constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 21;
static constexpr size_t kNoAllocStatsDoubles = 8;   // energy statistics, then the partials
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of g_noalloc_scratch per device.  In host code the symbol's name is only
// a host-side stand-in, so the address is looked up once per device with that device
// current, and the kernels receive the looked-up pointer.  The cached address belongs to
// the device's primary context: a cudaDeviceReset by the host program invalidates it (the
// module may be placed elsewhere afterwards), so this entry point must not be used on a
// device after a reset in the same process.
static constexpr int kMaxDevices = 64;
static double* g_scratch_ptr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

static cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace vmc

extern "C" vmc_status vmc_force_noalloc(const int8_t* spins, const float* tanh_theta,
                                        const float* eloc, int64_t n, int N, int M,
                                        double* F_out, double* meanO_out, void* stream) {
  using namespace vmc;
  if (!spins || !tanh_theta || !eloc || !F_out) return VMC_ERR_ARG;
  if (n < 1 || N < 1 || N > 1024 || M < 1 || M > 512) return VMC_ERR_ARG;
  const int64_t need = (int64_t)kNoAllocStatsDoubles + moments_partial_doubles(n, N, M);
  if (need > (int64_t)kNoAllocScratchDoubles) return VMC_ERR_ARG;
  if ((n + 1023) / 1024 > kMomentsMaxChunks) return VMC_ERR_ARG;   // grid z limit
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return VMC_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float2* E = reinterpret_cast<const float2*>(eloc);
  // every word of the scratch that the kernels read is written earlier in this call
  // (statistics first, then one partial per chunk and tile), so nothing is cleared
  if (launch_estats(E, n, scratch, nullptr, st) != cudaSuccess) return VMC_ERR_CUDA;
  if (launch_moments(spins, reinterpret_cast<const float2*>(tanh_theta), E, scratch, n, N, M,
                     scratch + kNoAllocStatsDoubles, reinterpret_cast<double2*>(meanO_out),
                     reinterpret_cast<double2*>(F_out), st) != cudaSuccess)
    return VMC_ERR_CUDA;
  return VMC_OK;
}
