// cg_tc.cu -- the two sample-sum products of the matrix-free S~ v on the 5th-generation
// tensor cores (CG on the shifted S, section "Diagonal shift"; S itself is never formed).
//
// For a CG direction v = [v_a | v_b | V] (V the W block as an M x N matrix):
//   Ov:  u_q = sum_j t_qj (v_b,j + Z_qj) + Z_q,M - c,      Z = S_b V^T,  c = <O> . v
//        S_b = spins as BF16 (exact), V as real rows 2j / 2j+1 = Re / Im V_j plus rows
//        2M / 2M+1 = Re / Im v_a, each row a BF16 hi/lo pair: Z = S_b V_hi^T + S_b V_lo^T.
//   OhU: w_q = u_q - mean(u);  y_W[j][i] = sum_q conj(t_qj) w_q s_qi,  y_a[i] = sum_q w_q s_qi,
//        y_b[j] = sum_q conj(t_qj) w_q.  The product A B^T has A rows 2j / 2j+1 = Re / Im of
//        conj(t_qj) w_q and rows 2M / 2M+1 = Re / Im w_q (as BF16 hi/lo pairs, samples q
//        along K) and B = spins^T; A is never stored: warps of the kernel form each 128 x 64
//        tile from t and u in shared memory (128-byte swizzled, as TMA would write it), so
//        t is read from HBM once per product.
//
// Both kernels are warp-specialised (warp 0: TMA, warp 1: tcgen05.mma issue, warps 2-9:
// epilogue or operand formation), hand stages over through mbarriers, and bound every wait:
// on expiry the kernel records DEV_ERR_TIMEOUT, the roles leave their loops, copies and
// products in flight are waited for (bounded), the tensor memory is freed and the kernel
// returns.
#include <algorithm>

#include "tc_ptx.cuh"
#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

namespace cgtc {
constexpr int TILE = 128 * 64 * 2;              // 128 rows x 64 BF16 (one swizzle row each)
constexpr int THREADS = 64 + 32 * 8;            // TMA warp, MMA warp, eight worker warps
constexpr int WORKER_WARPS = 8;
constexpr int OV_EPI_WARPS = 16;                // Ov: four warps per TMEM lane quadrant
constexpr int OV_THREADS = 64 + 32 * OV_EPI_WARPS;
constexpr int TAIL = 1024;                      // barriers and small shared scalars
// Ov: a work item is 256 samples (two 128-row sub-tiles sharing every V stage); K = N <= 256
constexpr int OV_MAX_NKB = 4;
constexpr int OV_STAGES = 3;
constexpr int OV_A_BYTES = OV_MAX_NKB * 2 * TILE;
constexpr int OV_STAGE_BYTES = 2 * TILE;        // V hi, V lo (128 rows each)
constexpr int OV_SMEM = 1024 + OV_A_BYTES + OV_STAGES * OV_STAGE_BYTES + TAIL;
constexpr int OV_TMEM_COLS = 512;               // two buffers x two sub-tiles x 128 columns
// OhU: per stage B = spins^T (up to 256 rows) and the block's 64 values of u in shared
// memory; A (hi, lo) in tensor memory
constexpr int OH_STAGES = 4;
constexpr int OH_B_BYTES = 2 * TILE;
constexpr int OH_U_BYTES = 64 * 8;
constexpr int OH_STAGE_BYTES = OH_B_BYTES + 1024;         // stages stay 1024-byte aligned
constexpr int OH_SMEM = 1024 + OH_STAGES * OH_STAGE_BYTES + TAIL;
constexpr int OH_TMEM_COLS = 512;                         // accumulator + 4 A stages
static_assert(256 + OH_STAGES * 64 <= OH_TMEM_COLS, "tensor memory budget");
static_assert(OV_SMEM <= 232448 && OH_SMEM <= 232448, "shared memory budget");

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

using tc::split_pair;
using tc::warp_wait;
}  // namespace cgtc

// ---------------------------------------------------------------------------------------
// Ov.  Persistent: CTA b takes items b, b + grid, ...  Per item the two spin sub-tiles stay
// in shared memory (one slot per 64-wide K block, refilled for the next item as soon as the
// item's last product on that block completes) while the V tiles stream through a 3-stage
// ring; each 128-column tile of Z (64 hidden units, re/im interleaved) accumulates in one
// of two TMEM buffers, so the epilogue of one column tile overlaps the products of the
// next.  Epilogue warp e (2..9) owns TMEM lane quadrant e % 4 of sub-tile (e - 2) / 4: one
// sample per thread, whose row of t it loads from HBM (32 hidden units ahead of use).
// upart[b] = FP64 sum of u over the samples CTA b wrote.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(cgtc::OV_THREADS, 1)
k_cg_ov(const __grid_constant__ CUtensorMap map_s, const __grid_constant__ CUtensorMap map_vhi,
        const __grid_constant__ CUtensorMap map_vlo, const __grid_constant__ CUtensorMap map_t,
        int prefetch_t, int nkb, int nct, int64_t items,
        const float2* __restrict__ T, const float2* __restrict__ vb, const double* __restrict__ c,
        int M, int64_t n, float2* __restrict__ u, double2* __restrict__ upart,
        const int* __restrict__ done, unsigned* status) {
  using namespace tc;
  using namespace cgtc;
  if (*done) return;                                      // the CG iteration has converged
  extern __shared__ uint8_t gsm_raw[];
  uint8_t* smem = align1024(gsm_raw);
  uint8_t* Abuf = smem;                                   // [kb][sub] tiles
  uint8_t* Bbuf = smem + OV_A_BYTES;                      // [stage][hi, lo]
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bbuf + OV_STAGES * OV_STAGE_BYTES);
  uint64_t* full = bars;                                  // [3] V stage landed
  uint64_t* empty = bars + 3;                             // [3] V stage consumed
  uint64_t* afull = bars + 6;                             // [4] spin slot landed
  uint64_t* aempty = bars + 10;                           // [4] spin slot consumed
  uint64_t* accf = bars + 14;                             // [2] accumulator complete
  uint64_t* acce = bars + 16;                             // [2] accumulator drained
  uint64_t* fin = bars + 18;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 19);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double2* red = reinterpret_cast<double2*>(bars + 20);   // [16]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 19; ++s) mbar_init(smem_u32(&bars[s]), 1);
    mbar_init(smem_u32(&acce[0]), OV_EPI_WARPS);
    mbar_init(smem_u32(&acce[1]), OV_EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(OV_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int64_t g = 0;                                      // V stages issued
      int last_it = -1, last_kb = -1;                     // the last spin slot load issued
      bool ok = true;
      int it = 0;
      for (int64_t w = blockIdx.x; w < items && ok && !*abort_flag; w += gridDim.x, ++it) {
        for (int kb = 0; kb < nkb && ok; ++kb) {
          if (it > 0 && !mbar_wait(smem_u32(&aempty[kb]), (uint32_t)((it - 1) & 1), abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&afull[kb]);
          mbar_expect_tx(fb, 2 * TILE);
          tma_load_2d(smem_u32(Abuf + (2 * kb) * TILE), &map_s, kb * 64, (int)(w * 256), fb);
          tma_load_2d(smem_u32(Abuf + (2 * kb + 1) * TILE), &map_s, kb * 64, (int)(w * 256 + 128), fb);
          last_it = it;
          last_kb = kb;
        }
        for (int ct = 0; ct < nct && ok; ++ct) {
          // t of this column tile's 256 samples into L2: the epilogue reads it one or two
          // column tiles from now
          if (prefetch_t) tma_prefetch_2d(&map_t, ct * 64, (int)(w * 256));
          for (int kb = 0; kb < nkb; ++kb, ++g) {
            const int s = (int)(g % OV_STAGES);
            if (g >= OV_STAGES &&
                !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((g / OV_STAGES) - 1) & 1), abort_flag)) {
              ok = false;
              break;
            }
            uint8_t* st = Bbuf + s * OV_STAGE_BYTES;
            const uint32_t fb = smem_u32(&full[s]);
            mbar_expect_tx(fb, 2 * TILE);
            tma_load_2d(smem_u32(st), &map_vhi, kb * 64, ct * 128, fb);
            tma_load_2d(smem_u32(st + TILE), &map_vlo, kb * 64, ct * 128, fb);
          }
        }
      }
      if (*abort_flag) {
        // copies in flight land before the CTA exits (bounded)
        volatile int dummy = 0;
        for (int64_t h = (g > OV_STAGES ? g - OV_STAGES : 0); h < g; ++h)
          mbar_wait(smem_u32(&full[h % OV_STAGES]), (uint32_t)((h / OV_STAGES) & 1), &dummy);
        for (int kb = 0; kb < nkb; ++kb) {
          const int cnt = (kb <= last_kb) ? last_it + 1 : last_it;   // loads into slot kb
          if (cnt > 0) mbar_wait(smem_u32(&afull[kb]), (uint32_t)((cnt - 1) & 1), &dummy);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t idesc = idesc_bf16_f32(128, 128);
      int64_t g = 0, cc = 0;
      bool ok = true, any = false;
      int it = 0;
      for (int64_t w = blockIdx.x; w < items && ok && !*abort_flag; w += gridDim.x, ++it) {
        for (int ct = 0; ct < nct && ok; ++ct, ++cc) {
          const int b = (int)(cc & 1);
          if (cc >= 2 && !mbar_wait(smem_u32(&acce[b]), (uint32_t)(((cc >> 1) - 1) & 1), abort_flag)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d0 = tmem + (uint32_t)(b * 256), d1 = d0 + 128u;
          for (int kb = 0; kb < nkb; ++kb, ++g) {
            if (ct == 0 && !mbar_wait(smem_u32(&afull[kb]), (uint32_t)(it & 1), abort_flag)) {
              ok = false;
              break;
            }
            const int s = (int)(g % OV_STAGES);
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((g / OV_STAGES) & 1), abort_flag)) {
              ok = false;
              break;
            }
            fence_after();
            const uint64_t a0 = smem_desc_sw128(smem_u32(Abuf + (2 * kb) * TILE));
            const uint64_t a1 = smem_desc_sw128(smem_u32(Abuf + (2 * kb + 1) * TILE));
            const uint64_t bh = smem_desc_sw128(smem_u32(Bbuf + s * OV_STAGE_BYTES));
            const uint64_t bl = smem_desc_sw128(smem_u32(Bbuf + s * OV_STAGE_BYTES + TILE));
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t o = (uint64_t)(kk * 32) >> 4;   // 16 BF16 = 32 bytes along K
              const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
              mma_bf16(d0, a0 + o, bh + o, idesc, acc);
              mma_bf16(d0, a0 + o, bl + o, idesc, 1u);
              mma_bf16(d1, a1 + o, bh + o, idesc, acc);
              mma_bf16(d1, a1 + o, bl + o, idesc, 1u);
            }
            any = true;
            mma_commit(smem_u32(&empty[s]));
            if (ct == nct - 1) mma_commit(smem_u32(&aempty[kb]));   // slot free for the next item
          }
          if (!ok) break;
          mma_commit(smem_u32(&accf[b]));
        }
      }
      if (*abort_flag && any) {
        volatile int dummy = 0;
        mma_commit(smem_u32(fin));
        mbar_wait(smem_u32(fin), 0, &dummy);
      }
    }
  } else {
    // ---------------- epilogue: u_q ----------------
    // Sixteen warps, four per TMEM lane quadrant (warp % 4): warp e reads lanes
    // 32 (e % 4) + 16 hh .. + 15 of sample sub-tile sub, (sub, hh) = ((e - 2) / 8, (e - 2) / 4 % 2),
    // with the 16x256b shape, one quarter (16 units = 32 columns) at a time: thread t gets
    // samples t/4 and t/4 + 8 of those 16 lanes and units 4 (t%4) .. + 3 of the quarter (the
    // V rows are ordered for this), so its t and v_b come in 16-byte loads; the four threads
    // of a sample sum their parts at the end of the item.
    const int ew = warp - 2;
    const int qd = warp & 3, sub = ew >> 3, hh = (ew >> 2) & 1;
    const int cq = lane & 3, sl = lane >> 2;
    const bool vec = (M & 1) == 0;
    const float cre = (float)c[0], cim = (float)c[1];
    const int row0 = sub * 128 + qd * 32 + 16 * hh + sl;    // sample of lane t/4 in the item
    // quarter (item w, column tile ct, qtr): units jb = 64 ct + 16 qtr ..; a quarter's t
    // (2 samples x 4 units per thread) is loaded two quarters ahead into one of three
    // rotating buffers; two cursors advance without divisions
    struct Cursor {
      int64_t w;
      int ct, qtr;
    };
    auto advance = [&](Cursor& k) {
      if (++k.qtr == 4) {
        k.qtr = 0;
        if (++k.ct == nct) {
          k.ct = 0;
          k.w += gridDim.x;
        }
      }
    };
    // dst[2 e + p]: units j0 + 2p, j0 + 2p + 1 of sample row0 + 8 e
    auto load_t = [&](const Cursor& k, float4 (&dst)[4]) {
      if (k.w >= items) return;
      const int j0 = k.ct * 64 + k.qtr * 16 + 4 * cq;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t m = k.w * 256 + row0 + 8 * e;
        if (m < n && vec && j0 + 4 <= M) {
          const float4* src = reinterpret_cast<const float4*>(T + m * M + j0);
          dst[2 * e] = src[0];
          dst[2 * e + 1] = src[1];
        } else {
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            const int j = j0 + 2 * p;
            const float2 x = (m < n && j < M) ? T[m * M + j] : make_float2(0.f, 0.f);
            const float2 y = (m < n && j + 1 < M) ? T[m * M + j + 1] : make_float2(0.f, 0.f);
            dst[2 * e + p] = make_float4(x.x, x.y, y.x, y.y);
          }
        }
      }
    };
    double usr = 0.0, usi = 0.0;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};    // [sample e][re, im]
    bool ok = true;
    int64_t cc = 0;                                 // column tiles completed
    Cursor use{(int64_t)blockIdx.x, 0, 0}, ahead = use;
    auto step = [&](const float4 (&cur)[4], float4 (&nxt)[4]) {
      if (!ok || use.w >= items) return;
      load_t(ahead, nxt);
      advance(ahead);
      const int b = (int)(cc & 1);
      if (use.qtr == 0) {
        if (!warp_wait(smem_u32(&accf[b]), (uint32_t)((cc >> 1) & 1), abort_flag, lane)) {
          ok = false;
          return;
        }
        fence_after();
      }
      const int j0 = use.ct * 64 + use.qtr * 16 + 4 * cq;
      float2 bv[4];
      if (j0 + 4 <= M) {
        const float4* vb4 = reinterpret_cast<const float4*>(vb + j0);
        const float4 x = vb4[0], y = vb4[1];
        bv[0] = make_float2(x.x, x.y);
        bv[1] = make_float2(x.z, x.w);
        bv[2] = make_float2(y.x, y.y);
        bv[3] = make_float2(y.z, y.w);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) bv[k] = (j0 + k < M) ? vb[j0 + k] : make_float2(0.f, 0.f);
      }
      const bool interior = j0 + 4 <= M;
      float v[16];
      tmem_ld16x256b_x4(tmem + ((uint32_t)(32 * qd + 16 * hh) << 16) +
                            (uint32_t)(b * 256 + sub * 128 + use.qtr * 32), v);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 t4 = cur[2 * e + (k >> 1)];
          const float tr = (k & 1) ? t4.z : t4.x, ti = (k & 1) ? t4.w : t4.y;
          const float zr0 = v[4 * k + 2 * e], zi0 = v[4 * k + 2 * e + 1];
          if (interior || j0 + k < M) {
            const float zr = zr0 + bv[k].x, zi = zi0 + bv[k].y;
            acc[e][0] = fmaf(tr, zr, fmaf(-ti, zi, acc[e][0]));
            acc[e][1] = fmaf(tr, zi, fmaf(ti, zr, acc[e][1]));
          } else if (j0 + k == M) {               // v_a rows: sum_i s_qi v_a,i as is
            acc[e][0] += zr0;
            acc[e][1] += zi0;
          }
        }
      }
      if (use.qtr == 3) {
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&acce[b]));
        ++cc;
        if (use.ct == nct - 1) {                   // the item's last column tile: u is complete
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            float xr = acc[e][0], xi = acc[e][1];
            xr += __shfl_xor_sync(0xffffffffu, xr, 1);
            xi += __shfl_xor_sync(0xffffffffu, xi, 1);
            xr += __shfl_xor_sync(0xffffffffu, xr, 2);
            xi += __shfl_xor_sync(0xffffffffu, xi, 2);
            const int64_t m = use.w * 256 + row0 + 8 * e;
            if (cq == 0 && m < n) {
              const float ur = xr - cre, ui = xi - cim;
              u[m] = make_float2(ur, ui);
              usr += (double)ur;
              usi += (double)ui;
            }
            acc[e][0] = acc[e][1] = 0.f;
          }
        }
      }
      advance(use);
    };
    float4 ta[4], tb[4], tc3[4];
    load_t(ahead, ta);
    advance(ahead);
    load_t(ahead, tb);
    advance(ahead);
    while (ok && use.w < items) {
      step(ta, tc3);
      step(tb, ta);
      step(tc3, tb);
    }
    usr = warp_sum_d(usr);
    usi = warp_sum_d(usi);
    if (lane == 0) red[ew] = make_double2(usr, usi);
    named_bar_sync(1, 32 * OV_EPI_WARPS);
    if (ew == 0 && lane == 0) {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < OV_EPI_WARPS; ++k) {
        sr += red[k].x;
        si += red[k].y;
      }
      upart[blockIdx.x] = make_double2(sr, si);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(OV_TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) flag_error(status, DEV_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------------------
// OhU.  CTA (mt, kc): rows [128 mt, 128 mt + 128) of A (hidden units 64 mt ..), K blocks
// [kc nkpc, ...) of the samples.  A is formed in tensor memory, never in shared memory:
// worker thread r (lane r of its warp's TMEM quadrant) owns row 2j + c of the tile and, for
// its half of each 64-sample block, loads t_qj of 32 samples (the warp's lanes cover 16
// consecutive units, so each load instruction reads 128 contiguous bytes of one sample's
// row), forms component c of conj(t_qj) w_q as a BF16 hi/lo pair and stores the packed
// pairs into the block's TMEM stage (tcgen05.st); the MMA takes A from TMEM and B =
// spins^T from shared memory.  w_q = u_q - mean(u) arrives in shared memory beside each B
// stage (1-D bulk copy of u).  The same threads keep y_b's FP32 partial sums and finally
// drain the accumulator.  TMEM: accumulator columns [0, 256); A stage s at columns
// 256 + 64 s (32 hi, then 32 lo; column m holds samples 2m, 2m + 1 of the block).
// out[kc][128 mt + r][col] = the chunk's FP32 partial of A B^T; ybpart[kc][j] likewise.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(cgtc::THREADS, 1)
k_cg_ohu(const __grid_constant__ CUtensorMap map_b, const __grid_constant__ CUtensorMap map_t,
         int prefetch_t, int nbt, int nkb, int nkpc, int mtiles, const float2* __restrict__ T,
         const float2* __restrict__ u, const double2* __restrict__ upart, int nup,
         const double* __restrict__ mean_in, int M, int64_t n, float* __restrict__ out,
         float2* __restrict__ ybpart, const int* __restrict__ done, unsigned* status) {
  using namespace tc;
  using namespace cgtc;
  if (*done) return;                                      // the CG iteration has converged
  extern __shared__ uint8_t gsm_raw[];
  uint8_t* smem = align1024(gsm_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OH_STAGES * OH_STAGE_BYTES);
  uint64_t* fullb = bars;                                 // [4] B and u landed
  uint64_t* fulla = bars + OH_STAGES;                     // [4] A formed (8 warps)
  uint64_t* empty = bars + 2 * OH_STAGES;                 // [4] stage consumed
  uint64_t* accf = bars + 3 * OH_STAGES;
  uint64_t* fin = accf + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float2* mean = reinterpret_cast<float2*>(fin + 2);

  const int mt = (int)(blockIdx.x % mtiles), kc = (int)(blockIdx.x / mtiles);
  const int kb0 = kc * nkpc, nk = min(nkb, kb0 + nkpc) - kb0;
  const int ncols = nbt * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 3 * OH_STAGES + 2; ++s) mbar_init(smem_u32(&bars[s]), 1);
    for (int s = 0; s < OH_STAGES; ++s) mbar_init(smem_u32(&fulla[s]), WORKER_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(OH_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (B = spins^T and u; t of later blocks into L2) ----------
      constexpr int PF = 4;                               // blocks of t prefetched ahead
      if (prefetch_t)
        for (int h = 0; h < PF && h < nk; ++h) tma_prefetch_2d(&map_t, mt * 64, (kb0 + h) * 64);
      int g = 0;
      for (; g < nk; ++g) {
        if (prefetch_t && g + PF < nk) tma_prefetch_2d(&map_t, mt * 64, (kb0 + g + PF) * 64);
        const int s = g % OH_STAGES;
        if (g >= OH_STAGES &&
            !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((g / OH_STAGES) - 1) & 1), abort_flag))
          break;
        uint8_t* st = smem + s * OH_STAGE_BYTES;
        const uint32_t fb = smem_u32(&fullb[s]);
        mbar_expect_tx(fb, (uint32_t)(nbt * TILE + OH_U_BYTES));
        for (int bt = 0; bt < nbt; ++bt)
          tma_load_2d(smem_u32(st + bt * TILE), &map_b, (kb0 + g) * 64, bt * 128, fb);
        bulk_load(smem_u32(st + OH_B_BYTES), u + (int64_t)(kb0 + g) * 64, OH_U_BYTES, fb);
      }
      if (*abort_flag) {
        volatile int dummy = 0;
        for (int h = (g > OH_STAGES ? g - OH_STAGES : 0); h < g; ++h)
          mbar_wait(smem_u32(&fullb[h % OH_STAGES]), (uint32_t)((h / OH_STAGES) & 1), &dummy);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = idesc_bf16_f32(128, ncols);
      bool any = false, ok = true;
      for (int g = 0; g < nk; ++g) {
        const int s = g % OH_STAGES;
        const uint32_t par = (uint32_t)((g / OH_STAGES) & 1);
        if (!mbar_wait(smem_u32(&fullb[s]), par, abort_flag) ||
            !mbar_wait(smem_u32(&fulla[s]), par, abort_flag)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t ah = tmem + (uint32_t)(256 + 64 * s), al = ah + 32u;
        const uint64_t bd = smem_desc_sw128(smem_u32(smem + s * OH_STAGE_BYTES));
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t o = (uint64_t)(kk * 32) >> 4;    // 16 BF16 along K
          mma_bf16_ts(tmem, ah + 8u * kk, bd + o, idesc, (g > 0 || kk > 0) ? 1u : 0u);
          mma_bf16_ts(tmem, al + 8u * kk, bd + o, idesc, 1u);
        }
        any = true;
        mma_commit(smem_u32(&empty[s]));
      }
      if (ok && any) mma_commit(smem_u32(accf));
      if (*abort_flag && any) {
        volatile int dummy = 0;
        mma_commit(smem_u32(fin));
        mbar_wait(smem_u32(fin), 0, &dummy);
      }
    }
  } else {
    // ---------------- A in TMEM, y_b partials, then the accumulator ----------------
    // TMEM lane L of the tile holds row (j, c) with j = 64 mt + 8 (L / 16) + L % 8 and
    // c = (L / 8) % 2 (the row order of A is free: D follows it).  Worker warp e writes
    // lanes 32 (e % 4) + 16 ((e - 2) / 4) .. + 15 with the 16x256b shape: thread t owns unit
    // jl = t / 4 of the warp's eight, both components (lanes jl and jl + 8), and samples
    // 16 k + 4 (t % 4) .. + 3 (k = 0..3) of each 64-sample block.
    const int ew = warp - 2;
    const int qd = warp & 3, hsel = ew >> 2;
    const int jl = lane >> 2, cq = lane & 3;
    const int j = mt * 64 + 8 * (2 * qd + hsel) + jl;
    const bool jv = j < M, jw = j == M;
    const uint32_t st_base = (uint32_t)(32 * qd + 16 * hsel) << 16;
    if (ew == 0) {
      // mean(u): given, or from the Ov CTAs' FP64 partials (fixed order)
      double sr = 0.0, si = 0.0;
      for (int k = lane; k < nup; k += 32) {
        sr += upart[k].x;
        si += upart[k].y;
      }
      sr = warp_sum_d(sr);
      si = warp_sum_d(si);
      if (lane == 0)
        *mean = mean_in ? make_float2((float)mean_in[0], (float)mean_in[1])
                        : make_float2((float)(sr / (double)n), (float)(si / (double)n));
    }
    named_bar_sync(1, 32 * WORKER_WARPS);
    const float mr = mean->x, mi = mean->y;
    // t of this thread's 16 samples of block g (rows 2M / 2M+1 carry w itself: t = 1;
    // samples q >= n get t = 0, and u there is finite: zeroed once, only finite values)
    const int64_t ldT = M;
    auto load_blk = [&](int g, float2 (&dst)[16]) {
      if (g >= nk) return;
      const int64_t qb = (int64_t)(kb0 + g) * 64 + 4 * cq;
      if (jv && qb + 52 < n) {
        const float2* tp = T + qb * ldT + j;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int i = 0; i < 4; ++i) dst[4 * k + i] = tp[(16 * k + i) * ldT];
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int64_t q = qb + 16 * k + i;
            const bool q_ok = q < n;
            dst[4 * k + i] = (jv && q_ok) ? T[q * ldT + j]
                                          : make_float2((jw && q_ok) ? 1.f : 0.f, 0.f);
          }
      }
    };
    float ybr = 0.f, ybi = 0.f;
    bool ok = true;
    float2 tn[16];
    load_blk(0, tn);
    for (int g = 0; g < nk; ++g) {
      float2 tq[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) tq[k] = tn[k];
      load_blk(g + 1, tn);
      const int s = g % OH_STAGES;
      // B and u of block g landed, which also means the MMA is done with A stage s
      if (!warp_wait(smem_u32(&fullb[s]), (uint32_t)((g / OH_STAGES) & 1), abort_flag, lane)) {
        ok = false;
        break;
      }
      fence_after();
      const float4* us = reinterpret_cast<const float4*>(smem + s * OH_STAGE_BYTES + OH_B_BYTES);
      uint32_t hi[16], lo[16];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float ar[4], ai[4];
#pragma unroll
        for (int i2 = 0; i2 < 2; ++i2) {
          const float4 uq = us[8 * k + 2 * cq + i2];       // samples 16k + 4cq + 2 i2, + 1
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int i = 2 * i2 + e;
            const float wr = (e ? uq.z : uq.x) - mr, wi = (e ? uq.w : uq.y) - mi;
            const float2 t = tq[4 * k + i];
            ar[i] = fmaf(t.x, wr, t.y * wi);                 // conj(t) w
            ai[i] = fmaf(t.x, wi, -t.y * wr);
            ybr += ar[i];
            ybi += ai[i];
          }
        }
        split_pair(ar[0], ar[1], hi[4 * k], lo[4 * k]);
        split_pair(ar[2], ar[3], hi[4 * k + 1], lo[4 * k + 1]);
        split_pair(ai[0], ai[1], hi[4 * k + 2], lo[4 * k + 2]);
        split_pair(ai[2], ai[3], hi[4 * k + 3], lo[4 * k + 3]);
      }
      const uint32_t col = (uint32_t)(256 + 64 * s);
      tmem_st16x256b_x4(tmem + st_base + col, hi);
      tmem_st16x256b_x4(tmem + st_base + col + 32u, lo);
      tmem_wait_st();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&fulla[s]));
    }
    // y_b: the four sample groups of each unit (lane bits 0-1), one FP32 partial per chunk
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      ybr += __shfl_xor_sync(0xffffffffu, ybr, o);
      ybi += __shfl_xor_sync(0xffffffffu, ybi, o);
    }
    if (ok && cq == 0 && jv) ybpart[(int64_t)kc * M + j] = make_float2(ybr, ybi);
    // the accumulator: quadrant qd, column half hsel; D lane L holds row (j(L), c(L))
    if (ok && nk > 0 && warp_wait(smem_u32(accf), 0u, abort_flag, lane)) {
      fence_after();
      const int L = 32 * qd + lane;
      const int arow = 2 * (8 * (L >> 4) + (L & 7)) + ((L >> 3) & 1);
      float* orow = out + ((int64_t)kc * mtiles * 128 + (int64_t)mt * 128 + arow) * ncols;
      for (int c0 = hsel * (ncols / 2); c0 < (hsel + 1) * (ncols / 2); c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int k = 0; k < 32; k += 4)
          *reinterpret_cast<float4*>(orow + c0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(OH_TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) flag_error(status, DEV_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
CgTcShape cg_tc_shape(int N, int M, int64_t n) {
  CgTcShape sh{};
  sh.kN = (N + 63) / 64 * 64;
  sh.s_rows = (n + 255) / 256 * 256;
  sh.v_rows = (2 * (int64_t)M + 2 + 127) / 128 * 128;
  sh.ldK = (n + 63) / 64 * 64;
  sh.b_rows = (N + 127) / 128 * 128;
  sh.nbt = (N + 127) / 128;
  sh.mtiles = (int)sh.v_rows / 128;
  const int nkb = (int)(sh.ldK / 64);
  const int sms = (int)persistent_grid(1 << 20);
  int kch = std::max(1, std::min(nkb, sms / sh.mtiles));
  sh.nkpc = (nkb + kch - 1) / kch;
  sh.kchunks = (nkb + sh.nkpc - 1) / sh.nkpc;               // no empty chunk
  sh.ok = N >= 1 && sh.kN <= 64 * cgtc::OV_MAX_NKB && sh.nbt <= 2;
  return sh;
}

cudaError_t launch_cg_ov_tc(const __nv_bfloat16* Sb, const __nv_bfloat16* Vhi,
                            const __nv_bfloat16* Vlo, const CgTcShape& sh, const float2* T,
                            const float2* vb, const double* c, int M, int64_t n, float2* u,
                            double2* upart, int* nup, const int* done, unsigned* status,
                            cudaStream_t st) {
  if (!sh.ok) return cudaErrorNotSupported;
  CUtensorMap ms, mvh, mvl, mt;
  cudaError_t e;
  // L2 prefetch boxes of t (8-byte elements): 64 hidden units x 256 samples; the rows of an
  // odd M are not 16-byte aligned, so those shapes go without
  const int pf = (M % 2 == 0) && make_map_c64(&mt, T, n, M, 64, 256) == cudaSuccess;
  if (!pf) mt = CUtensorMap{};
  if ((e = make_map(&ms, Sb, sh.s_rows, sh.kN)) != cudaSuccess) return e;
  if ((e = make_map(&mvh, Vhi, sh.v_rows, sh.kN)) != cudaSuccess) return e;
  if ((e = make_map(&mvl, Vlo, sh.v_rows, sh.kN)) != cudaSuccess) return e;
  static bool attr = false;
  if (!attr) {
    if ((e = cudaFuncSetAttribute(k_cg_ov, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  cgtc::OV_SMEM)) != cudaSuccess)
      return e;
    attr = true;
  }
  const int64_t items = sh.s_rows / 256;
  const unsigned grid = persistent_grid(items);
  k_cg_ov<<<grid, cgtc::OV_THREADS, cgtc::OV_SMEM, st>>>(ms, mvh, mvl, mt, pf, (int)(sh.kN / 64),
                                                      (int)(sh.v_rows / 128), items, T, vb, c, M,
                                                      n, u, upart, done, status);
  *nup = (int)grid;
  return cudaGetLastError();
}

cudaError_t launch_cg_ohu_tc(const __nv_bfloat16* Bs, const CgTcShape& sh, const float2* T,
                             const float2* u, const double2* upart, int nup, const double* mean,
                             int M, int64_t n, float* out, float2* ybpart, const int* done,
                             unsigned* status, cudaStream_t st) {
  if (!sh.ok) return cudaErrorNotSupported;
  CUtensorMap mb, mt;
  cudaError_t e;
  if ((e = make_map(&mb, Bs, sh.b_rows, sh.ldK)) != cudaSuccess) return e;
  // L2 prefetch boxes of t: 64 hidden units x 64 samples (none for an odd M)
  const int pf = (M % 2 == 0) && make_map_c64(&mt, T, n, M, 64, 64) == cudaSuccess;
  if (!pf) mt = CUtensorMap{};
  static bool attr = false;
  if (!attr) {
    if ((e = cudaFuncSetAttribute(k_cg_ohu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  cgtc::OH_SMEM)) != cudaSuccess)
      return e;
    attr = true;
  }
  const unsigned grid = (unsigned)(sh.mtiles * sh.kchunks);
  k_cg_ohu<<<grid, cgtc::THREADS, cgtc::OH_SMEM, st>>>(mb, mt, pf, sh.nbt, (int)(sh.ldK / 64), sh.nkpc,
                                                       sh.mtiles, T, u, upart, nup, mean, M, n, out,
                                                       ybpart, done, status);
  return cudaGetLastError();
}

}  // namespace vmc
