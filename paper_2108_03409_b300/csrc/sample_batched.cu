// sample_batched.cu -- every chain of many lattices of uneven size in one persistent
// launch, plus the per-lattice launcher that picks the model's sampler kernel.
#include "rbm_warp.cuh"

namespace vmc {

cudaError_t launch_sample_tfim(const SampleArgs& A, cudaStream_t st);
cudaError_t launch_sample_heis(const SampleArgs& A, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// Batched persistent sampler: many lattices (uneven N, M) in one launch.  Work items are
// (lattice, chain) pairs, ordered by the host so that the most expensive lattices come
// first; every warp takes the next item from an atomic counter until the list is done.
// The per-lattice arguments live in device memory (their sweep counters are advanced on
// the device after each call, so a captured graph can be replayed as is).  Blocks have at
// most 8 warps; the register budget (64 per thread up to four hidden slots per lane) keeps
// 32 warps resident per SM.
// ---------------------------------------------------------------------------------------
template <int MPL>
__global__ void __launch_bounds__(256, MPL <= 4 ? 4 : MPL <= 8 ? 3 : 2) k_sample_batched(const SampleArgs* __restrict__ args, const int* __restrict__ order,
                                 int n_lat, int C, int npad_max, unsigned* counter) {
  extern __shared__ int8_t sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int8_t* s = sm + wib * npad_max;
  const unsigned total = (unsigned)n_lat * (unsigned)C;
  while (true) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(counter, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    const int l = order[item / (unsigned)C];
    const int chain = (int)(item % (unsigned)C);
    const SampleArgs& A = args[l];
    if (A.lat.model == 1) run_chain<MPL, true>(A, chain, s, lane);
    else run_chain<MPL, false>(A, chain, s, lane);
    __syncwarp();
  }
}

__global__ void k_advance_sweeps(SampleArgs* args, int n_lat, uint64_t by) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n_lat) args[l].sweep0 += by;
}

cudaError_t launch_sample_batched(const SampleArgs* d_args, const int* d_order, int n_lat, int C,
                                  int Nmax, int Mmax, unsigned* counter, int warps_per_block,
                                  int grid, uint64_t advance, SampleArgs* d_args_mut,
                                  cudaStream_t st) {
  const int npad = (Nmax + 15) & ~15;
  const size_t smem = (size_t)warps_per_block * npad;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  VMC_DISPATCH_MPL(Mmax, k_sample_batched<MPL><<<grid, 32 * warps_per_block, smem, st>>>(
                             d_args, d_order, n_lat, C, npad, counter));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (advance) {
    k_advance_sweeps<<<(n_lat + 127) / 128, 128, 0, st>>>(d_args_mut, n_lat, advance);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

template <int MPL>
static int batched_occupancy(int threads, size_t smem) {
  int n = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sample_batched<MPL>, threads, smem) ==
                 cudaSuccess ? n : 0;
}

int batched_blocks_per_sm(int Mmax, int warps_per_block, int Nmax) {
  const size_t smem = (size_t)warps_per_block * ((Nmax + 15) & ~15);
  if (pick_mpl(Mmax) == 0) return 0;   // (the dispatch default below is then unreachable)
  auto occ = [&]() -> int {
    VMC_DISPATCH_MPL(Mmax, return batched_occupancy<MPL>(32 * warps_per_block, smem));
    return 0;
  };
  const int n = occ();
  return n > 0 ? n : 0;
}

cudaError_t launch_sample(const SampleArgs& A, cudaStream_t st) {
  return A.lat.model == 1 ? launch_sample_heis(A, st) : launch_sample_tfim(A, st);
}

}  // namespace vmc
