// vmc_device.cuh -- device helpers shared by the libvmc kernels: complex FP32 math for
// the RBM activations, the Philox4x64-10 counter RNG, lattice bonds and the device
// status word.  Internal to the library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vmc {

// ---------------------------------------------------------------------------------------
// device status word (bit flags, OR-ed by kernels, read at synchronising calls)
// ---------------------------------------------------------------------------------------
enum : unsigned {
  DEV_ERR_NUMERIC = 1u,   // non-finite value produced / non-positive pivot
  DEV_ERR_TIMEOUT = 2u,   // a bounded wait expired
  DEV_ERR_BOUNDS = 4u     // an index check failed (the access was skipped)
};

__device__ __forceinline__ void flag_error(unsigned* status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

// ---------------------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round multiplies
// counter words 0 and 2 by the published 64-bit multipliers, mixes the high halves with
// the other counter words and the key, and bumps the key by the Weyl constants.
// ---------------------------------------------------------------------------------------
struct u64x4 { uint64_t w0, w1, w2, w3; };

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                               uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  return {c0, c1, c2, c3};
}

// Map one Philox block to a Metropolis step: a uniform index in [0, K) from the top 32
// bits of word 0 (floor(r*K/2^32)), and u = (24-bit integer + 1/2) / 2^24 from word 1,
// returned as ln u.
__device__ __forceinline__ void mh_draw(const u64x4& w, uint32_t K, uint32_t* idx, float* logu) {
  uint32_t r = (uint32_t)(w.w0 >> 32);
  *idx = (uint32_t)(((uint64_t)r * (uint64_t)K) >> 32);
  float u = ((float)(uint32_t)(w.w1 >> 40) + 0.5f) * 5.9604644775390625e-08f;  // 2^-24
  *logu = logf(u);
}

// ---------------------------------------------------------------------------------------
// lattice
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ int num_bonds(int Lx, int Ly) {
  return Ly > 1 ? 2 * Lx * Ly : Lx * Ly;
}

__host__ __device__ __forceinline__ void bond_ends(int Lx, int Ly, int b, int* i, int* j) {
  const int N = Lx * Ly;
  const int site = b < N ? b : b - N;
  const int x = site % Lx, y = site / Lx;
  *i = site;
  *j = (b < N) ? ((x + 1) % Lx) + Lx * y : x + Lx * ((y + 1) % Ly);
}

// ---------------------------------------------------------------------------------------
// complex FP32 helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float reduce_angle(float y) {
  // y - 2 pi * rint(y / 2 pi), so that the fast sin/cos see |y| <= pi
  return fmaf(-6.28318530717958647692f, rintf(y * 0.15915494309189533577f), y);
}

// log cosh z = z' - ln 2 + log(1 + e^{-2 z'}), z' = +-z with Re z' >= 0.
__device__ __forceinline__ float2 logcosh_c(float x, float y) {
  if (x < 0.0f) { x = -x; y = -y; }
  float m = expf(-2.0f * x);
  float s, c;
  sincosf(-2.0f * y, &s, &c);
  float wr = m * c, wi = m * s;
  float re = x - 0.69314718055994531f + 0.5f * log1pf(fmaf(wr, wr, fmaf(wi, wi, 2.0f * wr)));
  float im = y + atan2f(wi, 1.0f + wr);
  return make_float2(re, im);
}

// tanh(x + iy) = (sinh 2x + i sin 2y) / (cosh 2x + cos 2y)
__device__ __forceinline__ float2 tanh_c(float x, float y) {
  if (fabsf(x) > 12.0f) return make_float2(copysignf(1.0f, x), 0.0f);
  float sh = sinhf(2.0f * x), ch = coshf(2.0f * x);
  float s, c;
  sincosf(2.0f * y, &s, &c);
  float d = ch + c;
  return make_float2(sh / d, s / d);
}

// complex division a / b
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  const float inv = 1.0f / fmaf(b.x, b.x, b.y * b.y);
  return make_float2(fmaf(a.x, b.x, a.y * b.y) * inv, fmaf(a.y, b.x, -a.x * b.y) * inv);
}

// Lower-triangular tile t of an nt x nt tile grid (bn <= bm), rasterised in groups of
// `group` tile rows and column-major inside a group, so that the tiles resident at the same
// time share a few row blocks of both operands.
__device__ __forceinline__ void grouped_tri_tile(int64_t t, int nt, int group, int* bm, int* bn) {
  // group index: the largest g with tri(group*g) <= t, tri(m) = m(m+1)/2
  int g = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5) / group;
  auto tri = [](int64_t m) { return m * (m + 1) / 2; };
  while (g > 0 && tri((int64_t)group * g) > t) --g;
  while (tri((int64_t)group * (g + 1)) <= t && group * (g + 1) < nt) ++g;
  const int r0 = group * g;
  const int r1 = min(r0 + group, nt) - 1;
  const int h = r1 - r0 + 1;
  int64_t u = t - tri(r0);
  if (u < (int64_t)r0 * h) {
    *bn = (int)(u / h);
    *bm = r0 + (int)(u % h);
    return;
  }
  u -= (int64_t)r0 * h;
  for (int c = r0; c <= r1; ++c) {
    const int height = r1 - c + 1;
    if (u < height) {
      *bn = c;
      *bm = c + (int)u;
      return;
    }
    u -= height;
  }
  *bm = r1;
  *bn = r1;
}

// Grid-wide barrier of a cooperative launch: a counter plus a generation word in global
// memory (zeroed before the launch).  Every wait is bounded (iteration and clock limits);
// an expired wait sets DEV_ERR_TIMEOUT and an abort word that makes every other block's
// wait give up too, so that all blocks leave their loops.  Returns false on abort.
struct GridBarrier {
  unsigned count;
  unsigned gen;
  unsigned abort;
};

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned nblocks, unsigned* status) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = &bar->gen;
    volatile unsigned* vab = &bar->abort;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const long long t0 = clock64();
      unsigned it = 0;
      while (*vgen == g) {
        if (*vab) { ok = 0; break; }
        if ((++it & 1023u) == 0 && clock64() - t0 > 2000000000ll) {
          atomicExch(&bar->abort, 1u);
          flag_error(status, DEV_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// warp reductions with xor butterflies: every lane ends with the same bits (each level
// adds the same two operands in both partner lanes).
// Compensated FP32 sum (Neumaier): s + c is the sum of the added FP32 values to within
// about one FP32 rounding of the result (plus count * 2^-48 of their magnitudes), with FP32
// operations only (on B300 an FP64 add per partial would bound the reduction on the FP64
// pipe).
struct CSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? (s - t) + v : (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A phase reduced to [-pi, pi]: y - k 2 pi with k = rint(y / 2 pi), the product k 2 pi
// taken in two FP32 parts (2 pi = C1 + C2, C1 the FP32 value nearest 2 pi; Cody and Waite's
// reduction) so that the result keeps FP32 accuracy for |k| up to a few thousand.
__device__ __forceinline__ float wrap_phase(float y) {
  const float k = rintf(y * 0.15915494309189533577f);
  y = fmaf(-k, 6.28318548202514648438f, y);
  return fmaf(k, 1.74845553146951715578e-7f, y);
}

// Warp sum of phases: every partial sum is reduced to [-pi, pi], so that a log psi whose
// imaginary part runs to many multiples of 2 pi (a Marshall sign, large weights) still has
// an absolute error of a few FP32 units of pi mod 2 pi.  Same bits in every lane.
__device__ __forceinline__ float warp_sum_phase(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = wrap_phase(v + __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace vmc
