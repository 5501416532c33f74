// sample_heis.cu -- Metropolis sampler kernel for the Heisenberg model (bond exchanges in the Sz = 0 sector);
// one warp per chain (the sweep itself is run_chain in rbm_warp.cuh).
#include "rbm_warp.cuh"

namespace vmc {

template <int MPL, bool HEIS>
__global__ void __launch_bounds__(128, sample_min_blocks(MPL)) k_sample(SampleArgs A) {
  extern __shared__ int8_t sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int chain = blockIdx.x * (blockDim.x >> 5) + wib;
  if (chain >= A.C) return;
  const int Npad = (A.rbm.N + 15) & ~15;
  run_chain<MPL, HEIS>(A, chain, sm + wib * Npad, lane, eloc_buffer(sm, A.rbm.N, wib));
}

cudaError_t launch_sample_heis(const SampleArgs& A, cudaStream_t st) {
  if (A.C <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((A.C + kWarps - 1) / kWarps);
  const size_t smem = sample_smem(A.rbm.N);
  VMC_DISPATCH_MPL(A.rbm.M, k_sample<MPL, true><<<grid, 32 * kWarps, smem, st>>>(A));
  return cudaGetLastError();
}

}  // namespace vmc
