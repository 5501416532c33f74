// cnn.cu -- the translation-symmetric single-layer CNN ansatz with ELU activation of the
// ground-state example (arXiv:2108.03409, section "Ground state search", Eq. gs_nqs):
//   log psi(s) = sum_a sum_r f_ELU(z_ar),  z_ar = sum_l W_al s_{(l+r) mod N} + b_a,
// real parameters, periodic chain, T = the N translations.  One warp per chain or sample;
// the alpha*N pre-activations z live in registers, entry e = a*N + r in slot e / 32 of lane
// e % 32.  A flip of site i changes z_ar by -2 s_i W_{a,(i-r) mod N}, so a proposal costs
// alpha*N ELU evaluations (no network re-evaluation); W sits in shared memory.
// Metropolis uses the RBM sampler's Philox stream and acceptance rule (mh_draw).
#include <cmath>

#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

namespace {

__device__ __forceinline__ float elu(float x) { return x > 0.f ? x : expm1f(x); }
__device__ __forceinline__ float delu(float x) { return x > 0.f ? 1.f : expf(x); }

// z of the warp's slots from the spins (shared memory) and W, b (shared memory)
template <int EPL>
__device__ __forceinline__ void cnn_preact(const CnnDev& D, const float* W, const float* b,
                                           const int8_t* s, int lane, float (&z)[EPL]) {
  const int N = D.N, E = D.alpha * N;
#pragma unroll
  for (int j = 0; j < EPL; ++j) {
    const int e = lane + 32 * j;
    float v = 0.f;
    if (e < E) {
      const int a = e / N, r = e % N;
      v = b[a];
      int idx = r;                                  // (l + r) mod N for l = 0, 1, ...
      for (int l = 0; l < N; ++l) {
        v = fmaf(W[a * N + l], (float)s[idx], v);
        idx = (idx + 1 == N) ? 0 : idx + 1;
      }
    }
    z[j] = v;
  }
}

template <int EPL>
__device__ __forceinline__ float cnn_sum_elu(const CnnDev& D, int lane, const float (&z)[EPL]) {
  const int E = D.alpha * D.N;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < EPL; ++j)
    if (lane + 32 * j < E) acc += elu(z[j]);
  return warp_sum(acc);
}

// log psi(s^(i)) - log psi(s) for the flip of site i (sign si = s_i)
template <int EPL>
__device__ __forceinline__ float cnn_flip_delta(const CnnDev& D, const float* W, int lane,
                                                const float (&z)[EPL], int i, float si) {
  const int N = D.N, E = D.alpha * N;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < EPL; ++j) {
    const int e = lane + 32 * j;
    if (e < E) {
      const int a = e / N, r = e % N;
      int l = i - r;
      if (l < 0) l += N;
      const float zn = fmaf(-2.f * si, W[a * N + l], z[j]);
      acc += elu(zn) - elu(z[j]);
    }
  }
  return warp_sum(acc);
}

template <int EPL>
__device__ float cnn_eloc(const CnnDev& D, const LatDev& L, const float* W, const int8_t* s,
                          int lane, const float (&z)[EPL]) {
  float zz = 0.f;
  for (int b = lane; b < L.nb; b += 32) {
    int i, j;
    bond_ends(L.Lx, L.Ly, b, &i, &j);
    zz += (float)(s[i] * s[j]);
  }
  zz = warp_sum(zz);
  float e = -L.J * zz;
  for (int i = 0; i < D.N; ++i) {
    const float d = cnn_flip_delta<EPL>(D, W, lane, z, i, (float)s[i]);
    e = fmaf(-L.h, expf(d), e);
  }
  return e;
}

// W and b into shared memory (block-wide)
__device__ __forceinline__ void cnn_stage(const CnnDev& D, float* W, float* b) {
  const int E = D.alpha * D.N;
  for (int k = threadIdx.x; k < E; k += blockDim.x) W[k] = D.W[k];
  for (int k = threadIdx.x; k < D.alpha; k += blockDim.x) b[k] = D.b[k];
  __syncthreads();
}

// Metropolis sweeps of every chain (one warp each): n_therm sweeps, then n_samples times
// (sweeps_per_sample sweeps, record spins / log psi / E_loc)
template <int EPL>
__global__ void __launch_bounds__(128) k_cnn_sample(CnnSampleArgs A) {
  extern __shared__ float csm[];
  const CnnDev& D = A.D;
  const int N = D.N, E = D.alpha * N;
  float* W = csm;
  float* b = W + E;
  int8_t* sbase = reinterpret_cast<int8_t*>(b + ((D.alpha + 3) & ~3));
  cnn_stage(D, W, b);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (c >= A.C) return;
  int8_t* s = sbase + wib * ((N + 15) & ~15);
  for (int i = lane; i < N; i += 32) s[i] = A.chains[c * N + i];
  __syncwarp();
  float z[EPL];
  cnn_preact<EPL>(D, W, b, s, lane, z);
  const int total = A.n_therm + A.n_samples * A.sweeps_per_sample;
  unsigned long long acc = 0;
  int rec = 0;
  for (int k = 0; k < total; ++k) {
    const uint64_t sweep = A.sweep0 + (uint64_t)k;
    for (int t0 = 0; t0 < A.L; t0 += 32) {
      // lane q draws step t0 + q
      uint32_t site_l = 0;
      float logu_l = 0.f;
      if (t0 + lane < A.L) {
        const u64x4 w = philox4x64_10((uint64_t)c, sweep, (uint64_t)(t0 + lane), 0ull, A.seed, A.stream);
        mh_draw(w, (uint32_t)N, &site_l, &logu_l);
      }
      const int steps = min(32, A.L - t0);
      for (int q = 0; q < steps; ++q) {
        const int i = (int)__shfl_sync(0xffffffffu, site_l, q);
        const float logu = __shfl_sync(0xffffffffu, logu_l, q);
        const float si = (float)s[i];
        const float d = cnn_flip_delta<EPL>(D, W, lane, z, i, si);
        if (logu < 2.f * d) {
#pragma unroll
          for (int j = 0; j < EPL; ++j) {
            const int e = lane + 32 * j;
            if (e < E) {
              const int a = e / N, r = e % N;
              int l = i - r;
              if (l < 0) l += N;
              z[j] = fmaf(-2.f * si, W[a * N + l], z[j]);
            }
          }
          __syncwarp();
          if (lane == 0) s[i] = (int8_t)(-s[i]);
          __syncwarp();
          ++acc;
        }
      }
    }
    if (k >= A.n_therm && (k - A.n_therm + 1) % A.sweeps_per_sample == 0) {
      cnn_preact<EPL>(D, W, b, s, lane, z);           // re-form z (removes the drift)
      const int64_t qs = (int64_t)rec * A.C + c;
      if (A.spins_out)
        for (int i = lane; i < N; i += 32) A.spins_out[qs * N + i] = s[i];
      if (A.logpsi_out) {
        const float lp = cnn_sum_elu<EPL>(D, lane, z);
        if (lane == 0) A.logpsi_out[qs] = lp;
      }
      if (A.eloc_out) {
        const float e = cnn_eloc<EPL>(D, A.lat, W, s, lane, z);
        if (lane == 0) {
          A.eloc_out[qs] = make_float2(e, 0.f);
          if (!isfinite(e)) flag_error(A.status, DEV_ERR_NUMERIC);
        }
      }
      ++rec;
    }
  }
  __syncwarp();
  for (int i = lane; i < N; i += 32) A.chains[c * N + i] = s[i];
  if (lane == 0 && A.n_accept) atomicAdd(A.n_accept, acc);
}

// log psi and (optionally) E_loc of given configurations, one warp each
template <int EPL>
__global__ void __launch_bounds__(128) k_cnn_eval(CnnDev D, LatDev L, const int8_t* __restrict__ spins,
                                                  int64_t n, float* __restrict__ logpsi,
                                                  float2* __restrict__ eloc, unsigned* status) {
  extern __shared__ float csm[];
  const int N = D.N, E = D.alpha * N;
  float* W = csm;
  float* b = W + E;
  int8_t* sbase = reinterpret_cast<int8_t*>(b + ((D.alpha + 3) & ~3));
  cnn_stage(D, W, b);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (q >= n) return;
  int8_t* s = sbase + wib * ((N + 15) & ~15);
  for (int i = lane; i < N; i += 32) s[i] = spins[q * N + i];
  __syncwarp();
  float z[EPL];
  cnn_preact<EPL>(D, W, b, s, lane, z);
  if (logpsi) {
    const float lp = cnn_sum_elu<EPL>(D, lane, z);
    if (lane == 0) logpsi[q] = lp;
  }
  if (eloc) {
    const float e = cnn_eloc<EPL>(D, L, W, s, lane, z);
    if (lane == 0) {
      eloc[q] = make_float2(e, 0.f);
      if (!isfinite(e)) flag_error(status, DEV_ERR_NUMERIC);
    }
  }
}

// dense O [n][P]: O_{W_al} = sum_r f'(z_ar) s_{(l+r) mod N}, O_{b_a} = sum_r f'(z_ar)
template <int EPL>
__global__ void __launch_bounds__(128) k_cnn_ok(CnnDev D, const int8_t* __restrict__ spins,
                                                int64_t n, float* __restrict__ O) {
  extern __shared__ float csm[];
  const int N = D.N, E = D.alpha * N;
  float* W = csm;
  float* b = W + E;
  float* dz_base = b + ((D.alpha + 3) & ~3);
  int8_t* sbase = reinterpret_cast<int8_t*>(dz_base + 4 * E);
  cnn_stage(D, W, b);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (q >= n) return;
  int8_t* s = sbase + wib * ((N + 15) & ~15);
  float* dz = dz_base + wib * E;
  for (int i = lane; i < N; i += 32) s[i] = spins[q * N + i];
  __syncwarp();
  float z[EPL];
  cnn_preact<EPL>(D, W, b, s, lane, z);
#pragma unroll
  for (int j = 0; j < EPL; ++j)
    if (lane + 32 * j < E) dz[lane + 32 * j] = delu(z[j]);
  __syncwarp();
  const int64_t P = (int64_t)E + D.alpha;
  for (int e = lane; e < E; e += 32) {             // entry (a, l)
    const int a = e / N, l = e % N;
    float v = 0.f;
    int idx = l;                                   // (l + r) mod N for r = 0, 1, ...
    for (int r = 0; r < N; ++r) {
      v = fmaf(dz[a * N + r], (float)s[idx], v);
      idx = (idx + 1 == N) ? 0 : idx + 1;
    }
    O[q * P + e] = v;
  }
  for (int a = lane; a < D.alpha; a += 32) {
    float v = 0.f;
    for (int r = 0; r < N; ++r) v += dz[a * N + r];
    O[q * P + E + a] = v;
  }
}

__global__ void k_cnn_prep(const double* p, int alpha, int N, float* W, float* b) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int E = alpha * N;
  if (k < E) W[k] = (float)p[k];
  else if (k < E + alpha) b[k - E] = (float)p[k];
}

// theta += dt Re(thetadot)
__global__ void k_cnn_update(double* p, const double2* td, int64_t P, double dt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < P) p[k] += dt * td[k].x;
}

#define CNN_DISPATCH(E, ...)                                          \
  do {                                                                \
    const int epl_ = ((E) + 31) / 32;                                 \
    if (epl_ <= 1) { constexpr int EPL = 1; __VA_ARGS__; }            \
    else if (epl_ <= 2) { constexpr int EPL = 2; __VA_ARGS__; }       \
    else if (epl_ <= 4) { constexpr int EPL = 4; __VA_ARGS__; }       \
    else if (epl_ <= 8) { constexpr int EPL = 8; __VA_ARGS__; }       \
    else if (epl_ <= 16) { constexpr int EPL = 16; __VA_ARGS__; }     \
    else return cudaErrorInvalidValue;                                \
  } while (0)

size_t cnn_smem(const CnnDev& D, bool with_dz) {
  const int E = D.alpha * D.N;
  return sizeof(float) * (E + ((D.alpha + 3) & ~3) + (with_dz ? 4 * E : 0)) +
         4 * (size_t)((D.N + 15) & ~15);
}

}  // namespace

cudaError_t launch_cnn_prep(const double* p, int alpha, int N, float* W, float* b, cudaStream_t st) {
  const int P = alpha * (N + 1);
  k_cnn_prep<<<(P + 255) / 256, 256, 0, st>>>(p, alpha, N, W, b);
  return cudaGetLastError();
}

cudaError_t launch_cnn_sample(const CnnSampleArgs& A, cudaStream_t st) {
  const int E = A.D.alpha * A.D.N;
  const unsigned grid = (unsigned)((A.C + 3) / 4);
  CNN_DISPATCH(E, k_cnn_sample<EPL><<<grid, 128, cnn_smem(A.D, false), st>>>(A));
  return cudaGetLastError();
}

cudaError_t launch_cnn_eval(const CnnDev& D, const LatDev& L, const int8_t* spins, int64_t n,
                            float* logpsi, float2* eloc, unsigned* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int E = D.alpha * D.N;
  const unsigned grid = (unsigned)((n + 3) / 4);
  CNN_DISPATCH(E, k_cnn_eval<EPL><<<grid, 128, cnn_smem(D, false), st>>>(D, L, spins, n, logpsi,
                                                                         eloc, status));
  return cudaGetLastError();
}

cudaError_t launch_cnn_ok(const CnnDev& D, const int8_t* spins, int64_t n, float* O, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int E = D.alpha * D.N;
  const unsigned grid = (unsigned)((n + 3) / 4);
  CNN_DISPATCH(E, k_cnn_ok<EPL><<<grid, 128, cnn_smem(D, true), st>>>(D, spins, n, O));
  return cudaGetLastError();
}

cudaError_t launch_cnn_update(double* p, const double2* td, int64_t P, double dt, cudaStream_t st) {
  k_cnn_update<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(p, td, P, dt);
  return cudaGetLastError();
}

}  // namespace vmc
