// sr.cu -- reductions of the SR/TDVP equation (Eq. qfm, Eq. force_vector):
// energy statistics, <O>, F, the centred log-derivative matrix and the FP32 Gram that
// gives S = <O^H O> - <O^H><O>.
#include <cstring>

#include <cuda_fp16.h>

#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

// ---------------------------------------------------------------------------------------
// energy statistics (FP64): mean, variance, naive standard error
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    t = warp_sum_d(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  return red[0];
}

__global__ void __launch_bounds__(1024) k_estats(const float2* __restrict__ E, int64_t n,
                                                 double* out, unsigned* status) {
  __shared__ double red[32];
  // per-thread sums in compensated FP32 (FP64 only across the block)
  CSum sr, si;
  bool bad = false;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
    float2 e = E[q];
    bad |= !isfinite(e.x) || !isfinite(e.y);
    sr.add(e.x);
    si.add(e.y);
  }
  const double mr = block_sum_d(sr.value(), red) / (double)n;
  const double mi = block_sum_d(si.value(), red) / (double)n;
  const float mrf = (float)mr, mif = (float)mi;
  const float cr = (float)(mr - (double)mrf), ci = (float)(mi - (double)mif);
  CSum v;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
    float2 e = E[q];
    const float dr = (e.x - mrf) - cr, di = (e.y - mif) - ci;
    v.add(fmaf(dr, dr, di * di));
  }
  const double var = block_sum_d(v.value(), red) / (double)n;
  if (threadIdx.x == 0) {
    out[0] = mr;
    out[1] = mi;
    out[2] = var;
    out[3] = sqrt(var / (double)n);
  }
  if (bad) flag_error(status, DEV_ERR_NUMERIC);
}

cudaError_t launch_estats(const float2* E, int64_t n, double* out, unsigned* status,
                          cudaStream_t st) {
  if (n <= 0) return cudaErrorInvalidValue;
  k_estats<<<1, 1024, 0, st>>>(E, n, out, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// <O> and F.  The index space is (j, i) in [0, M] x [0, N] with a virtual hidden unit
// j = M whose factor is 1 and a virtual visible unit i = N whose spin is 1:
//   (j < M, i < N): O = t_j s_i (W block);  (j < M, i = N): O = t_j (b block);
//   (j = M, i < N): O = s_i (a block).
// Each block sums a 32 x 16 tile over a chunk of kChunk samples: FP32 within sub-chunks of
// kSub samples, FP64 across them; chunk partials are then added in a fixed order.
// ---------------------------------------------------------------------------------------
static constexpr int kChunk = 1024, kSub = 128;
static_assert(kChunk == 8 * kSub, "one warp of the moments block per sub-chunk");

int64_t moments_partial_doubles(int64_t n, int N, int M) {
  int64_t chunks = (n + kChunk - 1) / kChunk;
  return chunks * 4 * (int64_t)(M + 1) * (N + 1);
}

// One block per (32 x 16 tile of the (i, j) index space, chunk of kChunk samples).  Warp w
// sums sub-chunk w of the chunk (kSub consecutive samples) in FP32; lane (li, lj) =
// (lane & 7, lane >> 3) holds the 4 x 4 entries i = i0 + 4 li + a, j = j0 + 4 lj + b and
// reads their spins, t and E itself (the tile's rows stay in L1 across the lanes that share
// them).  The warps' sub-chunk sums are then added in FP64 in sub-chunk order through
// shared memory, so a chunk's partial is the FP64 sum of its FP32 sub-chunk sums.
// WANT_M: also the sums of O (for <O>); without it only the F sums are formed (the CG
// operator's O^H u) and the <O> planes of the partials are left unwritten.
constexpr int MT_I = 32, MT_J = 16;

template <bool WANT_M>
__global__ void __launch_bounds__(256, 2) k_moments_partial(
    const int8_t* __restrict__ spins, const float2* __restrict__ T, const float2* __restrict__ E,
    const double* __restrict__ estats, int64_t n, int N, int M, double* __restrict__ partial) {
  constexpr int NPL = WANT_M ? 4 : 2;
  __shared__ double acc[NPL][MT_J][MT_I];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int li = lane & 7, lj = lane >> 3;
  const int ib = blockIdx.x * MT_I + 4 * li, jb = blockIdx.y * MT_J + 4 * lj;
  const int64_t q0 = (int64_t)blockIdx.z * kChunk + (int64_t)w * kSub;
  const int64_t q1 = min(n, q0 + kSub);
  const float emr = E ? (float)estats[0] : 0.f, emi = E ? (float)estats[1] : 0.f;
  float fr[4][4], fi[4][4], mr[4][4], mi[4][4];
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int a = 0; a < 4; ++a) fr[b][a] = fi[b][a] = mr[b][a] = mi[b][a] = 0.f;
#pragma unroll 2
  for (int64_t q = q0; q < q1; ++q) {
    float sv[4];
    float2 t[4], u[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = ib + a;
      sv[a] = (i < N) ? (float)spins[q * N + i] : (i == N ? 1.f : 0.f);
    }
    const float2 e = E ? E[q] : make_float2(0.f, 0.f);
    const float er = e.x - emr, ei = e.y - emi;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = jb + b;
      t[b] = (j < M) ? T[q * M + j] : make_float2(j == M ? 1.f : 0.f, 0.f);
      u[b] = make_float2(t[b].x * er + t[b].y * ei, t[b].x * ei - t[b].y * er);  // conj(t)(E-<E>)
    }
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (WANT_M) {
          mr[b][a] = fmaf(sv[a], t[b].x, mr[b][a]);
          mi[b][a] = fmaf(sv[a], t[b].y, mi[b][a]);
        }
        fr[b][a] = fmaf(sv[a], u[b].x, fr[b][a]);
        fi[b][a] = fmaf(sv[a], u[b].y, fi[b][a]);
      }
  }
  // FP64 sum over the sub-chunks, in order
  for (int k = 0; k < 8; ++k) {
    if (w == k) {
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int r = 4 * lj + b, c = 4 * li + a;
          const double v[4] = {(double)fr[b][a], (double)fi[b][a], (double)mr[b][a],
                               (double)mi[b][a]};
#pragma unroll
          for (int pl = 0; pl < NPL; ++pl)
            acc[pl][r][c] = (k == 0) ? v[pl] : acc[pl][r][c] + v[pl];
        }
    }
    __syncthreads();
  }
  // planes of the partials: 0, 1 = <O> sums (WANT_M), 2, 3 = F sums; acc planes 0, 1 hold
  // the F sums, 2, 3 the <O> sums
  const int64_t plane = (int64_t)(M + 1) * (N + 1);
  double* base = partial + (int64_t)blockIdx.z * 4 * plane;
  for (int e = threadIdx.x; e < MT_J * MT_I; e += 256) {
    const int r = e / MT_I, c = e % MT_I;
    const int j = blockIdx.y * MT_J + r, i = blockIdx.x * MT_I + c;
    if (i <= N && j <= M) {
      const int64_t off = (int64_t)j * (N + 1) + i;
      base[2 * plane + off] = acc[0][r][c];
      base[3 * plane + off] = acc[1][r][c];
      if (WANT_M) {
        base[off] = acc[2][r][c];
        base[plane + off] = acc[3][r][c];
      }
    }
  }
}

__global__ void k_moments_reduce(const double* __restrict__ partial, int64_t chunks, int64_t n,
                                 int N, int M, double2* __restrict__ meanO,
                                 double2* __restrict__ F) {
  const int64_t plane = (int64_t)(M + 1) * (N + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < plane;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / (N + 1)), i = (int)(e % (N + 1));
    if (j == M && i == N) continue;
    double m_r = 0, m_i = 0, f_r = 0, f_i = 0;
    for (int64_t c = 0; c < chunks; ++c) {
      const double* b = partial + c * 4 * plane + e;
      if (meanO) {
        m_r += b[0];
        m_i += b[plane];
      }
      f_r += b[2 * plane];
      f_i += b[3 * plane];
    }
    const double inv = 1.0 / (double)n;
    int64_t k;
    if (j == M) k = i;                                  // a block
    else if (i == N) k = N + j;                         // b block
    else k = (int64_t)N + M + (int64_t)j * N + i;       // W block
    if (meanO) meanO[k] = make_double2(m_r * inv, m_i * inv);
    if (F) F[k] = make_double2(f_r * inv, f_i * inv);
  }
}

cudaError_t launch_moments(const int8_t* spins, const float2* T, const float2* E,
                           const double* estats, int64_t n, int N, int M, double* partial,
                           double2* meanO, double2* F, cudaStream_t st) {
  if (n <= 0) return cudaErrorInvalidValue;
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  if (chunks > kMomentsMaxChunks) return cudaErrorInvalidValue;   // one chunk per grid z
  dim3 grid((N + 1 + MT_I - 1) / MT_I, (M + 1 + MT_J - 1) / MT_J, (unsigned)chunks);
  if (meanO) k_moments_partial<true><<<grid, 256, 0, st>>>(spins, T, E, estats, n, N, M, partial);
  else k_moments_partial<false><<<grid, 256, 0, st>>>(spins, T, E, estats, n, N, M, partial);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t plane = (int64_t)(M + 1) * (N + 1);
  int blocks = (int)std::min<int64_t>((plane + 255) / 256, 4096);
  k_moments_reduce<<<blocks, 256, 0, st>>>(partial, chunks, n, N, M, meanO, F);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// X = centred log-derivatives, transposed, real/imag rows interleaved, zero padded.
// One warp per (32 samples, hidden unit j); lane = sample.  The warp reads t_qj once and
// its sample's spins once (16-byte loads) and writes the rows of parameter b_j, of
// W_j1 .. W_jN and, for j < N, of a_j, 32 consecutive samples per store.  The mean is
// subtracted in FP32 as a hi/lo pair (o - m_hi - m_lo), which keeps the FP64 mean's
// accuracy in the centred value.
// ---------------------------------------------------------------------------------------
struct XOut {
  float* X32;
  __nv_bfloat16* Xhi;
  __nv_bfloat16* Xlo;
  __half* X16;                                   // one FP16 plane (the preconditioner's S)
  int64_t ld;
};

__device__ __forceinline__ void put_x(const XOut& o, int64_t k, int64_t q, float vr, float vi) {
  const int64_t r0 = (2 * k) * o.ld + q, r1 = r0 + o.ld;
  if (o.X32) {
    o.X32[r0] = vr;
    o.X32[r1] = vi;
  }
  if (o.Xhi) {
    const __nv_bfloat16 hr = __float2bfloat16_rn(vr), hi = __float2bfloat16_rn(vi);
    o.Xhi[r0] = hr;
    o.Xhi[r1] = hi;
    o.Xlo[r0] = __float2bfloat16_rn(vr - __bfloat162float(hr));
    o.Xlo[r1] = __float2bfloat16_rn(vi - __bfloat162float(hi));
  }
  if (o.X16) {
    o.X16[r0] = __float2half_rn(vr);
    o.X16[r1] = __float2half_rn(vi);
  }
}

// m = {Re hi, Im hi, Re lo, Im lo} of the FP64 mean
__device__ __forceinline__ float2 centre(float ox, float oy, float4 m) {
  return make_float2((ox - m.x) - m.z, (oy - m.y) - m.w);
}

__global__ void k_split_mean(const double2* __restrict__ meanO, int64_t P, float4* __restrict__ m2) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double2 m = meanO[k];
    const float hx = (float)m.x, hy = (float)m.y;
    m2[k] = make_float4(hx, hy, (float)(m.x - (double)hx), (float)(m.y - (double)hy));
  }
}

constexpr int BX_NMAX = 1024;

__global__ void __launch_bounds__(256) k_build_x(const int8_t* __restrict__ spins,
                                                 const float2* __restrict__ T,
                                                 const float4* __restrict__ meanO, int64_t n,
                                                 int N, int M, int64_t rows_pad, bool vec16,
                                                 XOut o) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.y * 8 + (threadIdx.x >> 5);
  const int64_t q = (int64_t)blockIdx.x * 32 + lane;
  if (j >= M || q >= o.ld) return;
  const bool live = q < n;
  const float2 t = live ? T[q * M + j] : make_float2(0.f, 0.f);
  // b_j
  {
    const int64_t k = N + j;
    float2 v = live ? centre(t.x, t.y, meanO[k]) : make_float2(0.f, 0.f);
    put_x(o, k, q, v.x, v.y);
  }
  // a_j (the first N warps of the j range)
  if (j < N) {
    const float sj = live ? (float)spins[q * N + j] : 0.f;
    float2 v = live ? centre(sj, 0.f, meanO[j]) : make_float2(0.f, 0.f);
    put_x(o, j, q, v.x, v.y);
  }
  // W_ji, i = 0 .. N-1 (rows N + M + j N + i)
  const int64_t kb = (int64_t)N + M + (int64_t)j * N;
  const int8_t* sq = spins + q * N;
  for (int i0 = 0; i0 < N; i0 += 16) {
    int8_t sv[16];
    if (live && vec16) {
      const int4 w = *reinterpret_cast<const int4*>(sq + i0);
      memcpy(sv, &w, 16);
    } else {
#pragma unroll
      for (int u = 0; u < 16; ++u) sv[u] = (live && i0 + u < N) ? sq[i0 + u] : (int8_t)0;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int i = i0 + u;
      if (i >= N) break;
      const float si = (float)sv[u];
      float2 v = live ? centre(si * t.x, si * t.y, meanO[kb + i]) : make_float2(0.f, 0.f);
      put_x(o, kb + i, q, v.x, v.y);
    }
  }
  // zero padding rows 2P .. rows_pad (written by the j = 0 warps)
  if (j == 0) {
    const int64_t P = (int64_t)N + M + (int64_t)N * M;
    for (int64_t k = P; 2 * k < rows_pad; ++k) put_x(o, k, q, 0.f, 0.f);
  }
}

cudaError_t launch_build_x(const int8_t* spins, const float2* T, const double2* meanO,
                           float4* mean2, int64_t n, int N, int M, int64_t rows_pad, int64_t ld,
                           float* X32, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, __half* X16,
                           cudaStream_t st) {
  if (N > BX_NMAX) return cudaErrorInvalidValue;
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  k_split_mean<<<(unsigned)std::min<int64_t>((P + 255) / 256, 1024), 256, 0, st>>>(meanO, P, mean2);
  dim3 grid((unsigned)((ld + 31) / 32), (unsigned)((M + 7) / 8));
  XOut o{X32, Xhi, Xlo, X16, ld};
  const bool vec16 = (N % 16) == 0 && (reinterpret_cast<uintptr_t>(spins) & 15) == 0;
  k_build_x<<<grid, 256, 0, st>>>(spins, T, mean2, n, N, M, rows_pad, vec16, o);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// FP32 SIMT Gram G = X X^T on lower-triangular 128x128 tiles (both operands have the
// sample index contiguous), 8x8 outputs per thread, double-buffered shared memory;
// the epilogue folds the 2x2 real blocks into complex S entries.
// ---------------------------------------------------------------------------------------
static constexpr int GB = 128, GK = 16, GPAD = 4;

__global__ void __launch_bounds__(256) k_gram_f32(const float* __restrict__ X, int64_t ld,
                                                  int nt, int64_t P, double inv_n,
                                                  double2* __restrict__ S, int mirror,
                                                  int ktpc, float2* __restrict__ part, int real) {
  extern __shared__ float gsm[];
  float* As = gsm;                              // [2][GK][GB + GPAD]
  float* Bs = gsm + 2 * GK * (GB + GPAD);       // [2][GK][GB + GPAD]
  int bm, bn;
  grouped_tri_tile(blockIdx.x, nt, 12, &bm, &bn);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float* Ag = X + (int64_t)bm * GB * ld;
  const float* Bg = X + (int64_t)bn * GB * ld;
  // K range of this block (blockIdx.y = sample chunk of ktpc GK-blocks)
  const int kt_begin = blockIdx.y * ktpc;
  const int ktiles = min((int)(ld / GK), kt_begin + ktpc) - kt_begin;
  Ag += (int64_t)kt_begin * GK;
  Bg += (int64_t)kt_begin * GK;

  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

  float4 ra[2], rb[2];
  auto gload = [&](int kt) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 256 * u;
      const int row = idx >> 2, c4 = idx & 3;
      ra[u] = *reinterpret_cast<const float4*>(Ag + (int64_t)row * ld + (int64_t)kt * GK + c4 * 4);
      rb[u] = *reinterpret_cast<const float4*>(Bg + (int64_t)row * ld + (int64_t)kt * GK + c4 * 4);
    }
  };
  auto sstore = [&](int buf) {
    float* a = As + buf * GK * (GB + GPAD);
    float* b = Bs + buf * GK * (GB + GPAD);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = tid + 256 * u;
      const int row = idx >> 2, c4 = idx & 3;
      a[(c4 * 4 + 0) * (GB + GPAD) + row] = ra[u].x;
      a[(c4 * 4 + 1) * (GB + GPAD) + row] = ra[u].y;
      a[(c4 * 4 + 2) * (GB + GPAD) + row] = ra[u].z;
      a[(c4 * 4 + 3) * (GB + GPAD) + row] = ra[u].w;
      b[(c4 * 4 + 0) * (GB + GPAD) + row] = rb[u].x;
      b[(c4 * 4 + 1) * (GB + GPAD) + row] = rb[u].y;
      b[(c4 * 4 + 2) * (GB + GPAD) + row] = rb[u].z;
      b[(c4 * 4 + 3) * (GB + GPAD) + row] = rb[u].w;
    }
  };

  gload(0);
  sstore(0);
  __syncthreads();
  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ktiles) gload(kt + 1);
    const float* a = As + buf * GK * (GB + GPAD);
    const float* b = Bs + buf * GK * (GB + GPAD);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float av[8], bv[8];
      float4 a0 = *reinterpret_cast<const float4*>(a + kk * (GB + GPAD) + ty * 4);
      float4 a1 = *reinterpret_cast<const float4*>(a + kk * (GB + GPAD) + ty * 4 + 64);
      float4 b0 = *reinterpret_cast<const float4*>(b + kk * (GB + GPAD) + tx * 4);
      float4 b1 = *reinterpret_cast<const float4*>(b + kk * (GB + GPAD) + tx * 4 + 64);
      av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
      av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
      bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
      bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
#pragma unroll
      for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
    }
    if (kt + 1 < ktiles) sstore(buf ^ 1);
    __syncthreads();
  }

  // epilogue: tile of G to shared memory, then fold 2x2 blocks into S
  float* Cs = gsm;  // [GB][GB + 1]
#pragma unroll
  for (int x = 0; x < 8; ++x) {
    const int r = (x < 4) ? ty * 4 + x : 64 + ty * 4 + (x - 4);
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const int c = (y < 4) ? tx * 4 + y : 64 + tx * 4 + (y - 4);
      Cs[r * (GB + 1) + c] = acc[x][y];
    }
  }
  __syncthreads();
  if (real) {
    // real rows (row k = parameter k): S_kl = G_kl / n, imaginary part 0
    for (int e = tid; e < GB * GB; e += 256) {
      const int r = e / GB, c = e % GB;
      const int64_t k = (int64_t)bm * GB + r, l = (int64_t)bn * GB + c;
      if (k >= P || l >= P || (bm == bn && l > k)) continue;
      const float g = Cs[r * (GB + 1) + c];
      if (part) {
        part[((int64_t)blockIdx.y * P + k) * P + l] = make_float2(g, 0.f);
        continue;
      }
      const double v = (double)g * inv_n;
      S[k * P + l] = make_double2(v, 0.0);
      if (mirror && l != k) S[l * P + k] = make_double2(v, 0.0);
    }
    return;
  }
  for (int e = tid; e < 64 * 64; e += 256) {
    const int r = e >> 6, c = e & 63;
    const int64_t k = (int64_t)bm * 64 + r, l = (int64_t)bn * 64 + c;
    if (k >= P || l >= P) continue;
    const float g00 = Cs[(2 * r) * (GB + 1) + 2 * c], g11 = Cs[(2 * r + 1) * (GB + 1) + 2 * c + 1];
    const float g01 = Cs[(2 * r) * (GB + 1) + 2 * c + 1], g10 = Cs[(2 * r + 1) * (GB + 1) + 2 * c];
    if (part) {
      if (bm != bn || l <= k)
        part[((int64_t)blockIdx.y * P + k) * P + l] = make_float2(g00 + g11, g01 - g10);
      continue;
    }
    const double re = ((double)g00 + (double)g11) * inv_n;
    const double im = ((double)g01 - (double)g10) * inv_n;
    S[k * P + l] = make_double2(re, im);
    if (mirror && bm != bn) S[l * P + k] = make_double2(re, -im);
  }
}

int gram_kchunks(int64_t tiles, int nkb, int64_t P, int64_t part_cap) {
  if (!part_cap || tiles >= 296) return 1;          // two waves of 148 SMs from tiles alone
  int64_t kc = std::min<int64_t>((296 + tiles - 1) / tiles, nkb / 16);
  kc = std::min<int64_t>(kc, part_cap / std::max<int64_t>(1, P * P));
  return (int)std::max<int64_t>(1, kc);
}

// S_kl = (1/n) sum over chunks (FP64) of the FP32 chunk folds, l <= k; mirrors as usual
__global__ void k_gram_reduce(const float2* __restrict__ part, int kchunks, int64_t P,
                              double inv_n, double2* __restrict__ S, float4* __restrict__ S2,
                              float2* __restrict__ Af, double nu, int shift_mode, int mirror) {
  const int64_t total = P * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / P, l = e - k * P;
    if (l > k) continue;
    double re = 0.0, im = 0.0;
    for (int c = 0; c < kchunks; ++c) {
      const float2 v = part[(int64_t)c * total + e];
      re += (double)v.x;
      im += (double)v.y;
    }
    const double vr = re * inv_n, vi = (l == k) ? 0.0 : im * inv_n;
    if (S) {
      S[e] = make_double2(vr, vi);
      if (mirror && l != k) S[l * P + k] = make_double2(vr, -vi);
    }
    if (S2 || Af) {
      const float hr = (float)vr, hi = (float)vi;
      if (S2) {
        S2[e] = make_float4(hr, hi, (float)(vr - (double)hr), (float)(vi - (double)hi));
        if (mirror && l != k) {
          const float mhi = (float)(-vi);
          S2[l * P + k] = make_float4(hr, mhi, (float)(vr - (double)hr), (float)(-vi - (double)mhi));
        }
      }
      if (Af) {
        const float d = (l == k) ? (float)(shift_mode == 0 ? vr * (1.0 + nu) : vr + nu) : hr;
        Af[e] = make_float2(d, hi);
      }
    }
  }
}

cudaError_t launch_gram_reduce(const float2* part, int kchunks, int64_t P, double inv_n,
                               double2* S, float4* S2, float2* Af, double nu, int shift_mode,
                               bool mirror, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((P * P + 255) / 256, 4096);
  k_gram_reduce<<<blocks, 256, 0, st>>>(part, kchunks, P, inv_n, S, S2, Af, nu, shift_mode,
                                        mirror ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_gram_f32(const float* X, int64_t rows_pad, int64_t ld, int64_t P,
                            double inv_n, double2* S, bool mirror, float2* part,
                            int64_t part_cap, cudaStream_t st, bool real) {
  if (rows_pad % GB != 0 || ld % GK != 0) return cudaErrorInvalidValue;
  const int64_t nt = rows_pad / GB;
  const int64_t tiles = nt * (nt + 1) / 2;
  const size_t smem = std::max<size_t>(2 * 2 * GK * (GB + GPAD) * sizeof(float),
                                       (size_t)GB * (GB + 1) * sizeof(float));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nkb = (int)(ld / 64);                    // chunk sizes in the 64-sample blocks
  int kchunks = gram_kchunks(tiles, nkb, P, part_cap);
  const int ktpc = ((nkb + kchunks - 1) / kchunks) * (64 / GK);
  kchunks = (int)((ld / GK + ktpc - 1) / ktpc);
  dim3 grid((unsigned)tiles, (unsigned)kchunks);
  k_gram_f32<<<grid, 256, smem, st>>>(X, ld, (int)nt, P, inv_n, S, mirror ? 1 : 0, ktpc,
                                      kchunks > 1 ? part : nullptr, real ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || kchunks == 1) return e;
  return launch_gram_reduce(part, kchunks, P, inv_n, S, nullptr, nullptr, 0.0, 0, mirror, st);
}

}  // namespace vmc
