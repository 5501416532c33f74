// sample_batched.cu -- every chain of many lattices of uneven size in one persistent
// launch, plus the per-lattice launcher that picks the model's sampler kernel.
#include "rbm_warp.cuh"

namespace vmc {

cudaError_t launch_sample_tfim(const SampleArgs& A, cudaStream_t st);
cudaError_t launch_sample_heis(const SampleArgs& A, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// Batched persistent sampler: many lattices (uneven N, M) in one launch.  A lattice's chains
// run in groups of G lanes (batched_group: 32 / G chains share a warp when its M hidden
// units fill G lanes' MPL slots), so that a small lattice does not pay a whole warp's
// reductions and bookkeeping per proposal.  Work units are one warp's chains of one
// lattice; ustart[o] is the first unit of the o-th lattice of the host's order (the most
// expensive lattices first), and every warp takes the next unit from an atomic counter
// until the list is done.  The per-lattice arguments live in device memory (their sweep
// counters are advanced on the device after each call, so a captured graph can be replayed
// as is).  Blocks have at most 8 warps; the register budget (64 per thread up to four
// hidden slots per lane) keeps 32 warps resident per SM.
// ---------------------------------------------------------------------------------------
template <int MPL, int G>
__device__ __forceinline__ void run_group(const SampleArgs& A, int chain, int8_t* s, int lane,
                                          float2* eb) {
  if (A.lat.model == 1) run_chain<MPL, true, G>(A, chain, s, lane, eb);
  else run_chain<MPL, false, G>(A, chain, s, lane, eb);
}

template <int MPL>
__global__ void __launch_bounds__(256, MPL <= 4 ? 4 : MPL <= 8 ? 3 : 2)
    k_sample_batched(const SampleArgs* __restrict__ args, const int* __restrict__ order,
                     const int* __restrict__ ustart, int n_lat, int npad_max, unsigned* counter) {
  extern __shared__ int8_t sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int8_t* sw = sm + wib * kMaxChainsPerWarp * npad_max;
  // the warp's local-energy ratio buffer (shared by its lane groups), after all warps' spin
  // buffers
  float2* eb = reinterpret_cast<float2*>(sm + (blockDim.x >> 5) * kMaxChainsPerWarp * npad_max +
                                         wib * kElocBufBytes);
  const unsigned total = (unsigned)ustart[n_lat];
  while (true) {
    unsigned unit = 0;
    if (lane == 0) unit = atomicAdd(counter, 1u);
    unit = __shfl_sync(0xffffffffu, unit, 0);
    if (unit >= total) break;
    int o = 0;
    while (o + 1 < n_lat && (unsigned)ustart[o + 1] <= unit) ++o;
    const SampleArgs& A = args[order[o]];
    const int G = (MPL <= 8) ? batched_group(A.rbm.M, MPL) : 32;
    const int gi = lane / G;
    const int chain = (int)(unit - (unsigned)ustart[o]) * (32 / G) + gi;
    if (chain < A.C) {
      int8_t* s = sw + gi * npad_max;
      if constexpr (MPL <= 8) {
        switch (G) {
          case 4: run_group<MPL, 4>(A, chain, s, lane, eb); break;
          case 8: run_group<MPL, 8>(A, chain, s, lane, eb); break;
          case 16: run_group<MPL, 16>(A, chain, s, lane, eb); break;
          default: run_group<MPL, 32>(A, chain, s, lane, eb); break;
        }
      } else {
        run_group<MPL, 32>(A, chain, s, lane, eb);
      }
    }
    __syncwarp();
  }
}

__global__ void k_advance_sweeps(SampleArgs* args, int n_lat, uint64_t by) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n_lat) args[l].sweep0 += by;
}

cudaError_t launch_sample_batched(const SampleArgs* d_args, const int* d_order,
                                  const int* d_ustart, int n_lat, int Nmax, int mpl,
                                  unsigned* counter, int warps_per_block, int grid,
                                  uint64_t advance, SampleArgs* d_args_mut, cudaStream_t st) {
  const int npad = (Nmax + 15) & ~15;
  const size_t smem = (size_t)warps_per_block * (kMaxChainsPerWarp * npad + kElocBufBytes);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  VMC_DISPATCH_MPL(32 * mpl, k_sample_batched<MPL><<<grid, 32 * warps_per_block, smem, st>>>(
                                 d_args, d_order, d_ustart, n_lat, npad, counter));
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

int batched_blocks_per_sm(int mpl, int warps_per_block, int Nmax) {
  const size_t smem = (size_t)warps_per_block * (kMaxChainsPerWarp * ((Nmax + 15) & ~15) + kElocBufBytes);
  if (pick_mpl(32 * mpl) != mpl) return 0;   // (the dispatch default below is then unreachable)
  auto occ = [&]() -> int {
    VMC_DISPATCH_MPL(32 * mpl, return batched_occupancy<MPL>(32 * warps_per_block, smem));
    return 0;
  };
  const int n = occ();
  return n > 0 ? n : 0;
}

int batched_chains_per_warp(int M, int mpl) {
  return mpl <= 8 ? 32 / batched_group(M, mpl) : 1;
}

int sample_slots_per_lane(int M) { return pick_mpl(M); }

cudaError_t launch_sample(const SampleArgs& A, cudaStream_t st) {
  return A.lat.model == 1 ? launch_sample_heis(A, st) : launch_sample_tfim(A, st);
}

}  // namespace vmc
