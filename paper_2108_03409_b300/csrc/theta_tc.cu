// theta_tc.cu -- theta = b + W s for a batch of configurations on the 5th-generation tensor
// cores (Eq. rbm_ex; the chains' theta at the start of an SR step, SURVEY's precision
// pattern: spins +-1 are exact in BF16, W is a BF16 hi + lo pair, FP32 accumulation).
//
// One CTA of eight warps forms a tile of 128 configurations x 64 hidden units:
//   D[q][2 jj + c] = sum_i s_qi part_c(W_{j0 + jj, i}),  c = 0 (Re), 1 (Im),
// a 128 x 128 real product accumulated in TMEM over 64-wide K blocks of the sites, two
// products per block (hi, lo).  The operands are written by the CTA into shared memory in the
// 128-byte-swizzled K-major layout the MMA descriptors name: the spins as BF16 (one 16-byte
// chunk per eight sites), W staged as [unit][site] and packed by rows 2 jj (Re) and
// 2 jj + 1 (Im).  The fold adds b and the tile is written through shared memory, coalesced.
// The MMA completion wait is bounded; on expiry the kernel records DEV_ERR_TIMEOUT, waits
// (bounded) for the products in flight, frees the tensor memory and returns.
#include "tc_ptx.cuh"
#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

namespace thtc {
constexpr int TQ = 128, TJ = 64, KB = 64;        // configurations, hidden units, sites per block
constexpr int OP = 128 * 128;                    // one operand plane: 128 rows x 128 bytes
constexpr int STG_LD = KB + 1;                   // W staging row stride (float2)
constexpr int OUT_LD = TJ + 1;                   // output staging row stride (float2)
constexpr int A_OFF = 0, BH_OFF = OP, BL_OFF = 2 * OP, STG_OFF = 3 * OP;
constexpr size_t SMEM = 1024 + 3 * OP + (size_t)TJ * STG_LD * 8;
static_assert((size_t)TQ * OUT_LD * 8 <= SMEM - 1024, "output staging fits");
constexpr int TMEM_COLS = 128;
}  // namespace thtc

__global__ void __launch_bounds__(256) k_theta_tc(const float2* __restrict__ b,
                                                  const float2* __restrict__ Wt, int N, int M,
                                                  const int8_t* __restrict__ spins, int64_t n,
                                                  float2* __restrict__ theta, unsigned* status) {
  using namespace thtc;
  extern __shared__ unsigned char raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) &
                                           ~uintptr_t(1023));
  __shared__ uint64_t bar[2];
  __shared__ uint32_t slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t q0 = (int64_t)blockIdx.x * TQ;
  const int j0 = blockIdx.y * TJ;
  float2* stg = reinterpret_cast<float2*>(sm + STG_OFF);
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(&bar[0]), 1);
    tc::mbar_init(tc::smem_u32(&bar[1]), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(tc::smem_u32(&slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = slot;
  const int nkb = (N + KB - 1) / KB;
  bool ok = true;
  uint32_t phase = 0;
  for (int kb = 0; kb < nkb && ok; ++kb) {
    const int i0 = kb * KB;
    // W of the tile's units over this block of sites, staged [unit][site] (coalesced reads
    // along the units of one site)
    for (int e = tid; e < TJ * KB; e += 256) {
      const int ii = e / TJ, jj = e % TJ;
      const int i = i0 + ii, j = j0 + jj;
      stg[jj * STG_LD + ii] = (i < N && j < M) ? Wt[(int64_t)i * M + j] : make_float2(0.f, 0.f);
    }
    // the spins as BF16 (+-1 exact, 0 beyond n and N): eight sites per 16-byte chunk
    for (int it = tid; it < TQ * 8; it += 256) {
      const int r = it >> 3, ch = it & 7;
      const int64_t q = q0 + r;
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = i0 + 8 * ch + 2 * e;
        const float s0 = (q < n && i < N) ? (float)spins[q * N + i] : 0.f;
        const float s1 = (q < n && i + 1 < N) ? (float)spins[q * N + i + 1] : 0.f;
        const __nv_bfloat162 h = __floats2bfloat162_rn(s0, s1);
        w[e] = *reinterpret_cast<const uint32_t*>(&h);
      }
      *reinterpret_cast<uint4*>(sm + A_OFF + tc::sw128_offset(r, ch)) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    // W as hi/lo planes: real rows 2 jj (Re), 2 jj + 1 (Im), eight sites per chunk
    for (int it = tid; it < TJ * 8; it += 256) {
      const int jj = it >> 3, ch = it & 7;
      const float2* src = stg + jj * STG_LD + 8 * ch;
      uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 x = src[2 * e], y = src[2 * e + 1];
        tc::split_pair(x.x, y.x, rh[e], rl[e]);
        tc::split_pair(x.y, y.y, ih[e], il[e]);
      }
      const uint32_t o0 = tc::sw128_offset(2 * jj, ch), o1 = tc::sw128_offset(2 * jj + 1, ch);
      *reinterpret_cast<uint4*>(sm + BH_OFF + o0) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
      *reinterpret_cast<uint4*>(sm + BL_OFF + o0) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
      *reinterpret_cast<uint4*>(sm + BH_OFF + o1) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
      *reinterpret_cast<uint4*>(sm + BL_OFF + o1) = make_uint4(il[0], il[1], il[2], il[3]);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 128);
      const uint64_t da = tc::smem_desc_sw128(tc::smem_u32(sm + A_OFF));
      const uint64_t dh = tc::smem_desc_sw128(tc::smem_u32(sm + BH_OFF));
      const uint64_t dl = tc::smem_desc_sw128(tc::smem_u32(sm + BL_OFF));
#pragma unroll
      for (int kk = 0; kk < KB / 16; ++kk) {
        const uint64_t o = (uint64_t)(kk * 32) >> 4;   // 16 BF16 along K
        tc::mma_bf16(tmem, da + o, dh + o, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        tc::mma_bf16(tmem, da + o, dl + o, idesc, 1u);
      }
      tc::mma_commit(tc::smem_u32(&bar[0]));
    }
    // the block's products must finish before its operands are overwritten (and, after the
    // last block, before the accumulator is read)
    const bool okw = tc::warp_wait(tc::smem_u32(&bar[0]), phase, &abort_flag, lane);
    phase ^= 1u;
    ok = __syncthreads_and(okw ? 1 : 0) != 0;
    tc::fence_after();
  }
  if (ok) {
    // fold: warp w reads TMEM lanes 32 (w % 4) .. (configurations) and columns 64 (w / 4) ..
    // (units 32 (w / 4) .. as Re/Im pairs); staged [configuration][unit] over the operands
    float2* out = reinterpret_cast<float2*>(sm);
    const int qd = warp & 3, hs = warp >> 2;
    const int r = 32 * qd + lane;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float d[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(64 * hs + 32 * h), d);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int jj = 32 * hs + 16 * h + u, j = j0 + jj;
        const float2 bj = (j < M) ? b[j] : make_float2(0.f, 0.f);
        out[r * OUT_LD + jj] = make_float2(d[2 * u] + bj.x, d[2 * u + 1] + bj.y);
      }
    }
    tc::fence_before();
    __syncthreads();
    for (int e = tid; e < TQ * TJ; e += 256) {
      const int rr = e / TJ, jj = e % TJ;
      const int64_t q = q0 + rr;
      const int j = j0 + jj;
      if (q < n && j < M) theta[q * M + j] = out[rr * OUT_LD + jj];
    }
  } else if (tid == 0) {
    flag_error(status, DEV_ERR_TIMEOUT);
    volatile int dummy = 0;                      // products in flight finish first (bounded)
    tc::mma_commit(tc::smem_u32(&bar[1]));
    tc::mbar_wait(tc::smem_u32(&bar[1]), 0, &dummy);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS) : "memory");
  }
}

cudaError_t launch_theta_tc(const RbmDev& R, const int8_t* spins, int64_t n, float2* theta,
                            unsigned* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_theta_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)thtc::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t gx = (n + thtc::TQ - 1) / thtc::TQ;
  if (gx > 2147483647) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gx, (unsigned)((R.M + thtc::TJ - 1) / thtc::TJ));
  if (grid.y > 65535) return cudaErrorInvalidValue;
  k_theta_tc<<<grid, 256, thtc::SMEM, st>>>(R.b, R.Wt, R.N, R.M, spins, n, theta, status);
  return cudaGetLastError();
}

}  // namespace vmc
