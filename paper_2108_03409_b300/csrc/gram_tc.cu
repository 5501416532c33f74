// gram_tc.cu -- S = <O^H O>^c (Eq. qfm) and the Schur-complement updates of the Cholesky
// factorisation on the 5th-generation tensor cores.
//
// The centred log-derivatives are stored as real rows X (row 2k = Re Obar_k, row 2k+1 =
// Im Obar_k, samples contiguous), split into BF16 pairs X = hi + lo.  The real Gram
// G = X X^T is accumulated in FP32 in tensor memory as hi.hi^T + hi.lo^T + lo.hi^T (the
// lo.lo^T term is 2^-16 below the others; PROD = 4 adds it), one 128 x 128 tile of G at a
// time, lower tiles only.  PROD = 1 takes X as one FP16 plane and one product: the S that
// only preconditions the SR step's CG (an 11-bit mantissa keeps the factor a good
// preconditioner at a third of the products).  The epilogue folds each 2x2 block of G into one complex entry:
//   S_kl = (G[2k][2l] + G[2k+1][2l+1] + i (G[2k][2l+1] - G[2k+1][2l])) / n.
//
// The kernel is persistent (one CTA per SM walks the tile list) and warp-specialised:
// warp 0 issues TMA loads (cp.async.bulk.tensor, 128-byte swizzle) into a ring of 3
// stages (6 for one FP16 plane, whose stages are half as large), warp 1 issues
// tcgen05.mma (kind::f16, BF16 or FP16 in, FP32 accumulate, 128 x 128 x 16) into one of two
// TMEM accumulators, and warps 2-9 (two per TMEM lane quadrant, each taking half of the
// columns) drain the other accumulator with tcgen05.ld, so
// the epilogue of one tile overlaps the loads and products of the next.  Ring stages and
// accumulators are handed over through mbarriers (tcgen05.commit arrives on them).  Every
// wait is bounded (iteration and clock limits); on expiry the kernel records
// DEV_ERR_TIMEOUT, every role leaves its loop, copies and products in flight are waited for
// (bounded), the tensor memory is freed and the kernel returns.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc_ptx.cuh"
#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;      // tile; BK = one 128-byte swizzle row of BF16
constexpr int STAGES = 3;                       // ring depth of the BF16 hi/lo products
constexpr int TILE_BYTES = BM * BK * 2;         // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;     // A_hi, A_lo, B_hi, B_lo
constexpr int RING_BYTES = STAGES * STAGE_BYTES;
// One FP16 plane needs half a stage, so the same ring holds twice the stages in flight
constexpr int MAX_STAGES = RING_BYTES / (2 * TILE_BYTES);
constexpr int STG_LD = 66;                      // staging row stride (float2) of the Schur epilogue
constexpr int STG_BYTES = 64 * STG_LD * 8;
constexpr int NUM_BARS = 2 * MAX_STAGES + 5;    // full, empty, acc full x2, acc empty x2, final
constexpr int SMEM_BYTES = 1024 /*align*/ + RING_BYTES + STG_BYTES + 256;
constexpr int EPI_WARPS = 8;                    // two per TMEM lane quadrant
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int THREADS = 64 + EPI_THREADS;       // TMA warp, MMA warp, 8 epilogue warps
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

}  // namespace tc

// Tile t of the lower triangle of nt x nt tiles (square 128 x 128 tiles).  tail > 0 (Schur updates): the tiles of
// the first tail tile columns -- the next panel's columns -- come last, column by column,
// so that they are the most recently written lines in L2 when the next panel starts.
__device__ __forceinline__ void schur_tile(int64_t t, int nt, int tail, int* bm, int* bn) {
  if (tail <= 0) {
    grouped_tri_tile(t, nt, 12, bm, bn);
    return;
  }
  const int n1 = nt - tail;
  const int64_t t1 = (int64_t)n1 * (n1 + 1) / 2;
  if (t < t1) {
    grouped_tri_tile(t, n1, 12, bm, bn);
    *bm += tail;
    *bn += tail;
    return;
  }
  int64_t u = t - t1;                  // column c < tail holds tile rows c .. nt - 1
  int c = 0;
  while (c < tail - 1 && u >= nt - c) {
    u -= nt - c;
    ++c;
  }
  *bn = c;
  *bm = c + (int)u;
}

// 128 x 256 tiles (BNT = 256): tile t is row tile bm = 2c + (t & 1) of the pair c and
// column tile bn <= c, with (c, bn) the lower triangle of the pairs walked as the square
// tiles are.  With an odd nt the pairs' last odd row lies past the operand (its boxes
// read the zero fill and the epilogue writes nothing for it).
__device__ __forceinline__ void wide_tile(int64_t t, int nt, int* bm, int* bn) {
  int c;
  grouped_tri_tile(t >> 1, (nt + 1) / 2, 6, &c, bn);
  *bm = 2 * c + (int)(t & 1);
}

template <int PROD, int BNT>
__global__ void __launch_bounds__(tc::THREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
          int nk, int nt, int64_t tiles, int64_t P, double inv_n, double2* __restrict__ S,
          float4* __restrict__ S2, float2* __restrict__ Af, double nu, int shift_mode, int mirror,
          float2* __restrict__ A32, int64_t ldA, int64_t off, int tail, int kchunks, int nkpc,
          float2* __restrict__ part, unsigned* status) {
  using namespace tc;
  extern __shared__ uint8_t gsm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) &
                                             ~uintptr_t(1023));
  // ring: PROD = 1 stages hold {A, B} (one FP16 plane; B is 256 rows when BNT = 256), the
  // others {A_hi, A_lo, B_hi, B_lo} of the BF16 products.  BNT = 256 serves only the S
  // Gram's factor-input epilogue (Af), with one sample chunk, and runs as clusters of two
  // CTAs on the row tiles 2c and 2c + 1 of one column tile: each CTA loads its own A and
  // one half of the shared B, which TMA writes into both CTAs' rings (this GPU's memory
  // only); a stage is free once both CTAs' products have read it.
  static_assert(BNT == BN || (BNT == 2 * BN && PROD == 1), "wide tiles: one FP16 plane only");
  constexpr bool PAIR = BNT != BN;
  constexpr int NST = PROD == 1 ? RING_BYTES / ((1 + BNT / BM) * TILE_BYTES) : STAGES;
  constexpr int SB = PROD == 1 ? (1 + BNT / BM) * TILE_BYTES : STAGE_BYTES;
  constexpr int TCOLS = 2 * BNT;                   // two accumulators of BNT columns
  constexpr int OFF_AL = TILE_BYTES, OFF_BH = PROD == 1 ? TILE_BYTES : 2 * TILE_BYTES,
                OFF_BL = 3 * TILE_BYTES;
  static_assert(NST * SB <= RING_BYTES, "ring");
  float2* stg = reinterpret_cast<float2*>(smem + RING_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RING_BYTES + STG_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + MAX_STAGES;
  uint64_t* accf = bars + 2 * MAX_STAGES;
  uint64_t* acce = bars + 2 * MAX_STAGES + 2;
  uint64_t* fin = bars + 2 * MAX_STAGES + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NUM_BARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // the epilogue leader's verdict per tile, in two slots by tile parity: a slot is rewritten
  // two tiles later, after every epilogue thread has passed the barrier that follows its read
  volatile int* epi_go = reinterpret_cast<volatile int*>(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NUM_BARS; ++s) mbar_init(smem_u32(&bars[s]), 1);
    mbar_init(smem_u32(&acce[0]), EPI_WARPS);
    mbar_init(smem_u32(&acce[1]), EPI_WARPS);
    if (PAIR)
      for (int s = 0; s < NST; ++s) mbar_init(smem_u32(&empty[s]), 2);   // both CTAs' products
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (PAIR) cluster_sync();                          // the peer's barriers are initialised
  const uint32_t crank = PAIR ? cluster_ctarank() : 0u;
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int64_t g = 0;                                  // k-blocks issued so far
      for (int64_t t = blockIdx.x; t < tiles * kchunks && !*abort_flag; t += gridDim.x) {
        int bm, bn;
        if (BNT == BN) schur_tile(t % tiles, nt, tail, &bm, &bn);
        else wide_tile(t, nt, &bm, &bn);
        const int kbeg = (int)(t / tiles) * nkpc, kend = min(nk, kbeg + nkpc);
        for (int kb = kbeg; kb < kend; ++kb, ++g) {
          const int s = (int)(g % NST);
          const int64_t j = g / NST;
          if (j > 0 && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((j - 1) & 1), abort_flag)) break;
          uint8_t* st = smem + s * SB;
          const uint32_t fb = smem_u32(&full[s]);
          mbar_expect_tx(fb, SB);
          tma_load_2d(smem_u32(st), &map_hi, kb * BK, bm * BM, fb);
          if (PROD != 1) tma_load_2d(smem_u32(st + OFF_AL), &map_lo, kb * BK, bm * BM, fb);
          if (PAIR)
            tma_load_2d_mc(smem_u32(st + OFF_BH + crank * TILE_BYTES), &map_hi, kb * BK,
                           bn * BNT + (int)crank * BN, fb, (uint16_t)3);
          else
            tma_load_2d(smem_u32(st + OFF_BH), &map_hi, kb * BK, bn * BNT, fb);
          if (PROD != 1) tma_load_2d(smem_u32(st + OFF_BL), &map_lo, kb * BK, bn * BN, fb);
        }
      }
      if (*abort_flag) {
        // let the copies in flight land before the CTA exits (bounded)
        volatile int dummy = 0;
        for (int64_t h = (g > NST ? g - NST : 0); h < g; ++h)
          mbar_wait(smem_u32(&full[h % NST]), (uint32_t)((h / NST) & 1), &dummy);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t idesc = PROD == 1 ? idesc_f16_f32(BM, BNT) : idesc_bf16_f32(BM, BNT);
      int64_t g = 0;
      int i = 0;
      bool issued_any = false;
      for (int64_t t = blockIdx.x; t < tiles * kchunks && !*abort_flag; t += gridDim.x, ++i) {
        const int acc = i & 1, u = i >> 1;
        if (u > 0 && !mbar_wait(smem_u32(&acce[acc]), (uint32_t)((u - 1) & 1), abort_flag)) break;
        fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * BNT);
        bool ok = true;
        const int kbeg = (int)(t / tiles) * nkpc, kend = min(nk, kbeg + nkpc);
        for (int kb = kbeg; kb < kend; ++kb, ++g) {
          const int s = (int)(g % NST);
          if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((g / NST) & 1), abort_flag)) { ok = false; break; }
          fence_after();
          uint8_t* st = smem + s * SB;
          const uint64_t ah = smem_desc_sw128(smem_u32(st));
          const uint64_t al = smem_desc_sw128(smem_u32(st + OFF_AL));
          const uint64_t bh = smem_desc_sw128(smem_u32(st + OFF_BH));
          const uint64_t bl = smem_desc_sw128(smem_u32(st + OFF_BL));
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t o = (uint64_t)(kk * 32) >> 4;   // 16 BF16 = 32 bytes along K
            mma_bf16(d, ah + o, bh + o, idesc, (kb > kbeg || kk > 0) ? 1u : 0u);
            if (PROD >= 3) {
              mma_bf16(d, ah + o, bl + o, idesc, 1u);
              mma_bf16(d, al + o, bh + o, idesc, 1u);
            }
            if (PROD == 4) mma_bf16(d, al + o, bl + o, idesc, 1u);   // (hi+lo)(hi+lo)^T: PSD
          }
          issued_any = true;
          if (PAIR) mma_commit_mc(smem_u32(&empty[s]), (uint16_t)3);   // in both CTAs
          else mma_commit(smem_u32(&empty[s]));        // frees the stage when these finish
        }
        if (!ok) break;
        mma_commit(smem_u32(&accf[acc]));              // accumulator complete
      }
      if (*abort_flag && issued_any) {
        // products in flight must finish before the tensor memory is freed (bounded)
        volatile int dummy = 0;
        mma_commit(smem_u32(fin));
        mbar_wait(smem_u32(fin), 0, &dummy);
      }
    }
  } else {
    // ------- epilogue: warps 2-9; TMEM lane quadrant = warp % 4, column half by warp -------
    const int qd = warp & 3;
    const int half = (warp - 2) >> 2;                // warps 2-5: first half of the columns
    const int r = qd * 32 + lane;                    // tile row held by this thread
    const int et = (warp - 2) * 32 + lane;           // 0..255 within the epilogue group
    const bool even = (r & 1) == 0;
    int i = 0;
    for (int64_t t = blockIdx.x; t < tiles * kchunks; t += gridDim.x, ++i) {
      const int acc = i & 1, u = i >> 1;
      int bm, bn;
      if (BNT == BN) schur_tile(t % tiles, nt, tail, &bm, &bn);
      else wide_tile(t, nt, &bm, &bn);
      const int kc = (int)(t / tiles);
      // Schur mode: fetch this thread's 16 entries of the factor's tile now, so that their
      // memory latency overlaps the wait for the products (no stores intervene).
      constexpr int PER = 64 * 64 / EPI_THREADS;
      float2 cur[PER];
      if (BNT == BN && A32) {
        const int64_t kb0 = (int64_t)bm * (BM / 2), lb0 = (int64_t)bn * (BN / 2);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
          const int e = et + EPI_THREADS * j, rr = e >> 6, cc = e & 63;
          const int64_t kk = kb0 + rr, ll = lb0 + cc;
          cur[j] = (kk < P && ll < P && (bm != bn || ll <= kk)) ? A32[(off + kk) * ldA + off + ll]
                                                              : make_float2(0.f, 0.f);
        }
      }
      if (et == 0)
        epi_go[i & 1] = mbar_wait(smem_u32(&accf[acc]), (uint32_t)(u & 1), abort_flag) && !*abort_flag;
      named_bar_sync(1, EPI_THREADS);                // the leader's verdict is uniform
      if (!epi_go[i & 1]) break;
      fence_after();
      const int64_t k = (int64_t)bm * (BM / 2) + (r >> 1);
      const float inv_nf = (float)inv_n, nuf = (float)nu;
      for (int c0 = half * (BNT / 2); c0 < (half + 1) * (BNT / 2); c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(acc * BNT + c0), v);
        const int64_t l0 = (int64_t)bn * (BNT / 2) + (c0 >> 1);
        if (BNT == BN && A32) {
          // Schur update: stage the fold (FP32) of this row pair; the even row keeps the
          // even q, the odd row the odd q.
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float mine0 = v[2 * q], mine1 = v[2 * q + 1];
            const float oth0 = __shfl_xor_sync(0xffffffffu, mine0, 1);
            const float oth1 = __shfl_xor_sync(0xffffffffu, mine1, 1);
            if ((q & 1) == (even ? 0 : 1)) {
              const float re = even ? mine0 + oth1 : oth0 + mine1;
              const float im = even ? mine1 - oth0 : oth1 - mine0;
              stg[(r >> 1) * STG_LD + (c0 >> 1) + q] = make_float2(re, im);
            }
          }
        } else if (BNT == BN && part) {
          // split over K: this chunk's fold (FP32, unnormalised) for l <= k; the chunks
          // are summed in FP64 afterwards
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float mine0 = v[2 * q], mine1 = v[2 * q + 1];
            const float oth0 = __shfl_xor_sync(0xffffffffu, mine0, 1);
            const float oth1 = __shfl_xor_sync(0xffffffffu, mine1, 1);
            const int64_t l = l0 + q;
            if (even && k < P && l < P && (bm != bn || l <= k))
              part[((int64_t)kc * P + k) * P + l] = make_float2(mine0 + oth1, mine1 - oth0);
          }
        } else if (Af && !S && !S2) {
          // the factor input alone (the preconditioner's S): FP32 arithmetic throughout --
          // an FP64 fold per entry would bound the tile on B300's FP64 pipe
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float mine0 = v[2 * q], mine1 = v[2 * q + 1];
            const float oth0 = __shfl_xor_sync(0xffffffffu, mine0, 1);
            const float oth1 = __shfl_xor_sync(0xffffffffu, mine1, 1);
            const int64_t l = l0 + q;
            if (even && k < P && l < P && l <= k) {
              const float vr = (mine0 + oth1) * inv_nf;
              const float vi = (l == k) ? 0.f : (mine1 - oth0) * inv_nf;
              Af[k * P + l] = make_float2(
                  (l == k) ? (shift_mode == 0 ? vr * (1.f + nuf) : vr + nuf) : vr, vi);
            }
          }
        } else {
          // row 2k holds G[2k][2l], G[2k][2l+1]; row 2k+1 holds G[2k+1][2l], G[2k+1][2l+1].
          // Off-diagonal tiles: the even row writes S_kl, the odd row its mirror.  In a
          // diagonal tile the accumulation order of (k,l) and (l,k) differs, so only l <= k
          // is taken and mirrored, which keeps S exactly Hermitian.
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float mine0 = v[2 * q], mine1 = v[2 * q + 1];
            const float oth0 = __shfl_xor_sync(0xffffffffu, mine0, 1);
            const float oth1 = __shfl_xor_sync(0xffffffffu, mine1, 1);
            const double re = even ? (double)mine0 + (double)oth1 : (double)oth0 + (double)mine1;
            const double im = even ? (double)mine1 - (double)oth0 : (double)oth1 - (double)mine0;
            const int64_t l = l0 + q;
            if (k < P && l < P && l <= k) {
              const double vr = re * inv_n, vi = (l == k) ? 0.0 : im * inv_n;
              if (even) {
                if (S) S[k * P + l] = make_double2(vr, vi);
                if (S2 || Af) {
                  const float hr = (float)vr, hi = (float)vi;
                  if (S2) S2[k * P + l] = make_float4(hr, hi, (float)(vr - (double)hr), (float)(vi - (double)hi));
                  if (Af) {
                    // the factor's input: lower triangle with the diagonal shift
                    const float d = (l == k) ? (float)(shift_mode == 0 ? vr * (1.0 + nu) : vr + nu) : hr;
                    Af[k * P + l] = make_float2(d, hi);
                  }
                }
              } else if (mirror && l != k) {
                if (S) S[l * P + k] = make_double2(vr, -vi);
                if (S2) {
                  const float hr = (float)vr, hi = (float)(-vi);
                  S2[l * P + k] = make_float4(hr, hi, (float)(vr - (double)hr), (float)(-vi - (double)hi));
                }
              }
            }
          }
        }
      }
      // the accumulator may be overwritten once every warp's loads have completed
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acce[acc]));
      if (BNT == BN && A32) {
        named_bar_sync(1, EPI_THREADS);              // staging complete
        // A[off+k][off+l] -= conj(fold) on l <= k, coalesced along rows; the diagonal
        // stays real.  (The next tile's writes to the staging buffer come after the next
        // named barrier, which every thread reaches only after this loop.)
        const int64_t kb0 = (int64_t)bm * (BM / 2), lb0 = (int64_t)bn * (BN / 2);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
          const int e = et + EPI_THREADS * j, rr = e >> 6, cc = e & 63;
          const int64_t kk = kb0 + rr, ll = lb0 + cc;
          if (kk < P && ll < P && (bm != bn || ll <= kk)) {
            const float2 f = stg[rr * STG_LD + cc];
            float2 a = cur[j];
            a.x -= f.x;
            if (ll != kk) a.y += f.y;
            A32[(off + kk) * ldA + off + ll] = a;
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  // the peer's copies into this CTA's ring and its products' arrivals on this CTA's
  // barriers are complete before either CTA of a pair exits
  if (PAIR) cluster_sync();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TCOLS) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) flag_error(status, DEV_ERR_TIMEOUT);
}

// Failure-path self-test: the tensor-core kernels' bounded mbarrier wait on a barrier that
// nothing arrives at must give up, set the abort flag and report DEV_ERR_TIMEOUT.
__global__ void k_selftest_mbar_wait(unsigned* status) {
  using namespace tc;
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!mbar_wait(smem_u32(&bar), 0, &abort_flag)) flag_error(status, DEV_ERR_TIMEOUT);
  }
}

cudaError_t launch_selftest_mbar_wait(unsigned* status, cudaStream_t st) {
  k_selftest_mbar_wait<<<1, 32, 0, st>>>(status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
// cuTensorMapEncodeTiled is a driver-API function; it is looked up through the runtime so
// that the library has no link-time dependency on libcuda (it still loads on machines
// without a GPU driver, where only argument checking is possible).
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* base, int64_t rows, int64_t ld) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = encode_tiled();
  if (!encode) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {tc::BK, tc::BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                      const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_map_c64(CUtensorMap* map, const float2* base, int64_t rows, int64_t cols,
                         int box_cols, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = encode_tiled();
  if (!encode) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 8};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<float2*>(base), dims,
                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// one CTA per SM (the kernels' shared memory allows no second one), at most one per tile
unsigned persistent_grid(int64_t tiles) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 148;
  }
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
}

static cudaError_t gram_attrs() {
  static bool attr = false;
  if (attr) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_gram_tc<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::SMEM_BYTES)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_gram_tc<1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::SMEM_BYTES)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_gram_tc<3, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::SMEM_BYTES)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_gram_tc<4, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::SMEM_BYTES)) != cudaSuccess)
    return e;
  attr = true;
  return cudaSuccess;
}

// Launch configuration of the paired (128 x 256 tile) kernel: clusters of two CTAs, as many
// clusters as fit on the GPU at once (each CTA takes a whole SM); grid 0 if none fit.
static cudaLaunchConfig_t pair_config(cudaLaunchAttribute* attr, int64_t pairs, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(tc::THREADS, 1, 1);
  cfg.dynamicSmemBytes = tc::SMEM_BYTES;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  static int clusters = -1;
  if (clusters < 0) {
    cfg.gridDim = dim3(2, 1, 1);
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, (const void*)k_gram_tc<1, 256>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      c = 0;
    }
    clusters = c;
  }
  cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(clusters, pairs)), 1, 1);
  return cfg;
}

// prod: 1 (one FP16 plane in Xhi, Xlo unused), 3 or 4 (BF16 hi/lo planes)
cudaError_t launch_gram_tc(const __nv_bfloat16* Xhi, const __nv_bfloat16* Xlo,
                           int64_t rows_pad, int64_t ld, int64_t P, double inv_n, double2* S,
                           bool mirror, float4* S2, float2* Af, double nu, int shift_mode,
                           int prod, float2* part, int64_t part_cap, unsigned* status,
                           cudaStream_t st) {
  if (rows_pad % tc::BM != 0 || ld % tc::BK != 0 || ld < tc::BK) return cudaErrorNotSupported;
  if (prod != 1 && prod != 3 && prod != 4) return cudaErrorInvalidValue;
  if (prod == 1) Xlo = Xhi;                          // (the map of an unused plane)
  if ((reinterpret_cast<uintptr_t>(Xhi) | reinterpret_cast<uintptr_t>(Xlo)) & 15)
    return cudaErrorNotSupported;
  CUtensorMap mhi, mlo;
  cudaError_t e;
  // the maps move 2-byte elements bit for bit: the same map serves BF16 and FP16 planes
  if ((e = make_map(&mhi, Xhi, rows_pad, ld)) != cudaSuccess) return e;
  if ((e = make_map(&mlo, Xlo, rows_pad, ld)) != cudaSuccess) return e;
  if ((e = gram_attrs()) != cudaSuccess) return e;
  const int64_t nt = rows_pad / tc::BM;
  const int64_t tiles = nt * (nt + 1) / 2;
  const int nkb = (int)(ld / tc::BK);
  int kchunks = gram_kchunks(tiles, nkb, P, part_cap);
  const int nkpc = (nkb + kchunks - 1) / kchunks;
  kchunks = (nkb + nkpc - 1) / nkpc;                 // no empty chunk
  if (prod == 1 && kchunks == 1 && Af && !S && !S2) {
    // the factor input alone from one FP16 plane: 128 x 256 tiles computed by CTA pairs
    // that share the B tile (each CTA loads 32 KB per 64 samples for a 128 x 256 block:
    // two thirds of the operand traffic of the 128 x 128 tiles per product)
    const int64_t ntc = (nt + 1) / 2, pairs = ntc * (ntc + 1) / 2;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair_config(attr, pairs, st);
    if (cfg.gridDim.x > 0) {
      double2* no_s = nullptr;
      float4* no_s2 = nullptr;
      float2* no_f2 = nullptr;
      return cudaLaunchKernelEx(&cfg, k_gram_tc<1, 256>, mhi, mlo, nkb, (int)nt, 2 * pairs, P,
                                inv_n, no_s, no_s2, Af, nu, shift_mode, 0, no_f2, (int64_t)0,
                                (int64_t)0, 0, 1, nkb, no_f2, status);
    }
  }
  auto kern = prod == 1 ? k_gram_tc<1, 128> : prod == 4 ? k_gram_tc<4, 128> : k_gram_tc<3, 128>;
  kern<<<persistent_grid(tiles * kchunks), tc::THREADS, tc::SMEM_BYTES, st>>>(
      mhi, mlo, nkb, (int)nt, tiles, P, inv_n, S, S2, Af, nu, shift_mode, mirror ? 1 : 0,
      nullptr, 0, 0, 0, kchunks, nkpc, kchunks > 1 ? part : nullptr, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (kchunks > 1)
    return launch_gram_reduce(part, kchunks, P, inv_n, S, S2, Af, nu, shift_mode, mirror, st);
  return cudaSuccess;
}

cudaError_t launch_herk_tc(const __nv_bfloat16* Xhi, const __nv_bfloat16* Xlo, int64_t rows_pad,
                           int64_t K, int64_t n, float2* A32, int64_t ldA, int64_t off,
                           int tail_cols, int prod, unsigned* status, cudaStream_t st) {
  if (rows_pad % tc::BM != 0 || K % tc::BK != 0 || K < tc::BK) return cudaErrorNotSupported;
  if (prod != 1 && prod != 3) return cudaErrorInvalidValue;
  if (prod == 1) Xlo = Xhi;
  CUtensorMap mhi, mlo;
  cudaError_t e;
  if ((e = make_map(&mhi, Xhi, rows_pad, K)) != cudaSuccess) return e;
  if ((e = make_map(&mlo, Xlo, rows_pad, K)) != cudaSuccess) return e;
  if ((e = gram_attrs()) != cudaSuccess) return e;
  const int64_t nt = rows_pad / tc::BM;
  const int64_t tiles = nt * (nt + 1) / 2;
  // the first tail_cols columns (128-row tiles of the real operand = 64 complex columns)
  // are updated last
  const int tail = (int)std::min<int64_t>(nt, std::max<int64_t>(0, (tail_cols + 63) / 64));
  auto kern = prod == 1 ? k_gram_tc<1, 128> : k_gram_tc<3, 128>;
  kern<<<persistent_grid(tiles), tc::THREADS, tc::SMEM_BYTES, st>>>(
      mhi, mlo, (int)(K / tc::BK), (int)nt, tiles, n, 1.0, nullptr, nullptr, nullptr, 0.0, 0, 0,
      A32, ldA, off, tail, 1, (int)(K / tc::BK), nullptr, status);
  return cudaGetLastError();
}

}  // namespace vmc
