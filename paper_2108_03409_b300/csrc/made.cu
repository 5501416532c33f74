// made.cu -- learned proposal: a masked autoregressive MLP q(s) (MADE; Germain, Gregor,
// Murray, Larochelle 2015) built on the paper's autoregressive factorisation
// p(s) = p1(s1) p2(s2|s1) ... (section "Autoregressive neural quantum states"), used for
// independent Metropolis-Hastings moves accepted with min(1, |psi(s')|^2 q(s) / |psi(s)|^2 q(s')).
//
// Network (degrees 1-based; hidden unit k of both layers has degree m(k) = (k mod (N-1)) + 1):
//   h1 = relu(W1 s + b1),  W1[k][d] used iff m(k) >= d
//   h2 = relu(W2 h1 + b2), W2[k2][k1] used iff m(k2) >= m(k1)
//   z  = W3 h2 + b3,       W3[d][k2] used iff d > m(k2);  q(s) = prod_d sigma(s_d z_d)
// Parameters (FP32 master copy, canonical layout) W1[H][N] | b1[H] | W2[H][H] | b2[H] |
// W3[N][H] | b3[N]; transposed copies W1t[N][H], W2t[H][H], W3t[H][N] keep every loop over
// a layer's inputs coalesced across the warp's lanes.
#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {


__device__ __forceinline__ int made_degree(int k, int N) { return (k % (N - 1)) + 1; }

__device__ __forceinline__ float log_sigmoid_f(float x) {
  return (x >= 0.f) ? -log1pf(expf(-x)) : x - log1pf(expf(x));
}

int64_t made_nparams(int N, int H) {
  return (int64_t)H * N + H + (int64_t)H * H + H + (int64_t)N * H + N;
}

MadeDev made_view(float* theta, float* W1t, float* W2t, float* W3t, int N, int H) {
  MadeDev D;
  D.N = N;
  D.H = H;
  D.W1 = theta;
  D.b1 = D.W1 + (int64_t)H * N;
  D.W2 = D.b1 + H;
  D.b2 = D.W2 + (int64_t)H * H;
  D.W3 = D.b2 + H;
  D.b3 = D.W3 + (int64_t)N * H;
  D.W1t = W1t;
  D.W2t = W2t;
  D.W3t = W3t;
  return D;
}

// refresh the transposed copies from the canonical weights
__global__ void k_made_transpose(MadeDev D) {
  const int N = D.N, H = D.H;
  const int64_t n1 = (int64_t)H * N, n2 = (int64_t)H * H;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n1 + n2 + n1;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < n1) {                       // W1[k][d] -> W1t[d][k]
      const int64_t k = e / N, d = e % N;
      const_cast<float*>(D.W1t)[d * H + k] = D.W1[e];
    } else if (e < n1 + n2) {           // W2[k2][k1] -> W2t[k1][k2]
      const int64_t f = e - n1, k2 = f / H, k1 = f % H;
      const_cast<float*>(D.W2t)[k1 * H + k2] = D.W2[f];
    } else {                            // W3[d][k2] -> W3t[k2][d]
      const int64_t f = e - n1 - n2, d = f / H, k2 = f % H;
      const_cast<float*>(D.W3t)[k2 * N + d] = D.W3[f];
    }
  }
}

// ---------------------------------------------------------------------------------------
// forward (and optionally the backward pass of the loss -(1/n) sum log q) for a batch,
// one warp per sample; lane l owns hidden units k = l + 32 j and logits d = l + 32 j.
// ---------------------------------------------------------------------------------------
template <int HPL>
__global__ void __launch_bounds__(128) k_made_fwd(MadeDev D, const int8_t* __restrict__ spins,
                                                  int64_t n, float* __restrict__ logq,
                                                  float* __restrict__ H1, float* __restrict__ H2,
                                                  float* __restrict__ G1, float* __restrict__ G2,
                                                  float* __restrict__ G3, float inv_batch) {
  extern __shared__ unsigned char msm[];
  const int N = D.N, H = D.H;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (q >= n) return;
  const int Npad = (N + 15) & ~15;
  float* h1 = reinterpret_cast<float*>(msm) + wib * (2 * H);
  float* h2 = h1 + H;
  int8_t* s = reinterpret_cast<int8_t*>(reinterpret_cast<float*>(msm) + (blockDim.x >> 5) * 2 * H) + wib * Npad;
  for (int i = lane; i < N; i += 32) s[i] = spins[q * N + i];
  __syncwarp();
  float a[HPL];
#pragma unroll
  for (int j = 0; j < HPL; ++j) a[j] = D.b1[lane + 32 * j];
  for (int d = 0; d < N; ++d) {
    const float sd = (float)s[d];
#pragma unroll
    for (int j = 0; j < HPL; ++j) {
      const int k = lane + 32 * j;
      if (made_degree(k, N) >= d + 1) a[j] = fmaf(D.W1t[(int64_t)d * H + k], sd, a[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < HPL; ++j) {
    const float v = fmaxf(a[j], 0.f);
    h1[lane + 32 * j] = v;
    if (H1) H1[q * H + lane + 32 * j] = v;
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < HPL; ++j) a[j] = D.b2[lane + 32 * j];
  for (int k1 = 0; k1 < H; ++k1) {
    const float hv = h1[k1];
    if (hv == 0.f) continue;                                   // uniform across the warp
    const int m1 = made_degree(k1, N);
#pragma unroll
    for (int j = 0; j < HPL; ++j) {
      const int k2 = lane + 32 * j;
      if (made_degree(k2, N) >= m1) a[j] = fmaf(D.W2t[(int64_t)k1 * H + k2], hv, a[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < HPL; ++j) {
    const float v = fmaxf(a[j], 0.f);
    h2[lane + 32 * j] = v;
    if (H2) H2[q * H + lane + 32 * j] = v;
  }
  __syncwarp();
  float lq = 0.f;
  for (int d = lane; d < N; d += 32) {
    float z = D.b3[d];
    for (int k2 = 0; k2 < H; ++k2) {
      const float hv = h2[k2];
      if (d + 1 > made_degree(k2, N)) z = fmaf(D.W3t[(int64_t)k2 * N + d], hv, z);
    }
    const float sd = (float)s[d];
    lq += log_sigmoid_f(sd * z);
    if (G3) G3[q * N + d] = -sd / (1.f + expf(sd * z)) * inv_batch;   // d(-log sigma(s z))/dz / n
  }
  lq = warp_sum(lq);
  if (lane == 0 && logq) logq[q] = lq;
  if (!G3) return;
  __syncwarp();
  // backward: g2[k2] = relu'(a2) sum_{d > m(k2)} W3[d][k2] g3[d]
  float g[HPL];
#pragma unroll
  for (int j = 0; j < HPL; ++j) g[j] = 0.f;
  for (int d = 0; d < N; ++d) {
    const float g3 = G3[q * N + d];
#pragma unroll
    for (int j = 0; j < HPL; ++j) {
      const int k2 = lane + 32 * j;
      if (d + 1 > made_degree(k2, N)) g[j] = fmaf(D.W3[(int64_t)d * H + k2], g3, g[j]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < HPL; ++j) {
    const int k2 = lane + 32 * j;
    const float v = (h2[k2] > 0.f) ? g[j] : 0.f;
    G2[q * H + k2] = v;
    h2[k2] = v;                                   // reuse: h2 now holds g2
  }
  __syncwarp();
  // g1[k1] = relu'(a1) sum_{k2: m(k2) >= m(k1)} W2[k2][k1] g2[k2]
#pragma unroll
  for (int j = 0; j < HPL; ++j) g[j] = 0.f;
  for (int k2 = 0; k2 < H; ++k2) {
    const float gv = h2[k2];
    if (gv == 0.f) continue;
    const int m2 = made_degree(k2, N);
#pragma unroll
    for (int j = 0; j < HPL; ++j) {
      const int k1 = lane + 32 * j;
      if (m2 >= made_degree(k1, N)) g[j] = fmaf(D.W2[(int64_t)k2 * H + k1], gv, g[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < HPL; ++j) {
    const int k1 = lane + 32 * j;
    G1[q * H + k1] = (h1[k1] > 0.f) ? g[j] : 0.f;
  }
}

// ---------------------------------------------------------------------------------------
// masked weight gradients C[i][j] = sum_b A[b][i] B[b][j] (FP32), 64 x 64 tiles
//   MODE 1: dW1[k1][d], A = G1 [n][H], B = spins [n][N], kept iff m(k1) >= d + 1
//   MODE 2: dW2[k2][k1], A = G2, B = H1, kept iff m(k2) >= m(k1)
//   MODE 3: dW3[d][k2],  A = G3 [n][N], B = H2, kept iff d + 1 > m(k2)
// ---------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_made_outer(const float* __restrict__ A,
                                                    const void* __restrict__ Bv, int64_t n,
                                                    int I, int J, int N, float* __restrict__ C) {
  __shared__ float As[32][64 + 1];
  __shared__ float Bs[32][64 + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int64_t b0 = 0; b0 < n; b0 += 32) {
    for (int e = tid; e < 32 * 64; e += 256) {
      const int bb = e / 64, c = e % 64;
      const int64_t b = b0 + bb;
      As[bb][c] = (b < n && i0 + c < I) ? A[b * I + i0 + c] : 0.f;
      float bv = 0.f;
      if (b < n && j0 + c < J) {
        if (MODE == 1) bv = (float)reinterpret_cast<const int8_t*>(Bv)[b * J + j0 + c];
        else bv = reinterpret_cast<const float*>(Bv)[b * J + j0 + c];
      }
      Bs[bb][c] = bv;
    }
    __syncthreads();
#pragma unroll 4
    for (int bb = 0; bb < 32; ++bb) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[bb][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[bb][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx + 16 * b;
      if (i >= I || j >= J) continue;
      bool keep;
      if (MODE == 1) keep = made_degree(i, N) >= j + 1;
      else if (MODE == 2) keep = made_degree(i, N) >= made_degree(j, N);
      else keep = i + 1 > made_degree(j, N);
      C[(int64_t)i * J + j] = keep ? acc[a][b] : 0.f;
    }
  }
}

// bias gradients: out[i] = sum_b A[b][i]
__global__ void k_made_colsum(const float* __restrict__ A, int64_t n, int I, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  float s = 0.f;
  for (int64_t b = 0; b < n; ++b) s += A[b * I + i];
  out[i] = s;
}

// Adam (Kingma & Ba 2014) with bias corrections c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
__global__ void k_adam(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int64_t np, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    th[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
  }
}

// ---------------------------------------------------------------------------------------
// Autoregressive sampling, one warp per sample, sites in order.  A hidden unit of degree m
// depends only on s_1..s_m, so it is evaluated once, right after site m is drawn; the
// logit of site d uses the second-layer units of degree < d.  Site d draws
//   u = ((w[(d-1) mod 4] >> 40) + 1/2) / 2^24,  w = Philox4x64-10({c, round, (d-1)/4, 2},
//   {seed, stream}),  s_d = +1 iff u < sigma(z_d).
// ---------------------------------------------------------------------------------------
template <int HPL>
__global__ void __launch_bounds__(128) k_made_sample(MadeDev D, int64_t n, uint64_t seed,
                                                     uint64_t stream, uint64_t round,
                                                     int8_t* __restrict__ spins,
                                                     float* __restrict__ logq) {
  extern __shared__ unsigned char msm[];
  const int N = D.N, H = D.H;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (c >= n) return;
  const int Npad = (N + 15) & ~15;
  float* h1 = reinterpret_cast<float*>(msm) + wib * (2 * H);
  float* h2 = h1 + H;
  int8_t* s = reinterpret_cast<int8_t*>(reinterpret_cast<float*>(msm) + (blockDim.x >> 5) * 2 * H) + wib * Npad;
  float a[HPL];
#pragma unroll
  for (int j = 0; j < HPL; ++j) {
    a[j] = D.b1[lane + 32 * j];
    h1[lane + 32 * j] = 0.f;
    h2[lane + 32 * j] = 0.f;
  }
  __syncwarp();
  float lq = 0.f;
  u64x4 w = {0, 0, 0, 0};
  for (int d = 1; d <= N; ++d) {
    // logit of site d from the second-layer units of degree < d
    float zp = 0.f;
#pragma unroll
    for (int j = 0; j < HPL; ++j) {
      const int k2 = lane + 32 * j;
      if (made_degree(k2, N) < d) zp = fmaf(D.W3[(int64_t)(d - 1) * H + k2], h2[k2], zp);
    }
    const float z = warp_sum(zp) + D.b3[d - 1];
    if (((d - 1) & 3) == 0) w = philox4x64_10((uint64_t)c, round, (uint64_t)((d - 1) >> 2), 2ull, seed, stream);
    const uint64_t wd = ((d - 1) & 3) == 0 ? w.w0 : ((d - 1) & 3) == 1 ? w.w1 : ((d - 1) & 3) == 2 ? w.w2 : w.w3;
    const float u = ((float)(uint32_t)(wd >> 40) + 0.5f) * 5.9604644775390625e-08f;
    const float p = 1.f / (1.f + expf(-z));
    const float sd = (u < p) ? 1.f : -1.f;
    lq += log_sigmoid_f(sd * z);
    if (lane == 0) s[d - 1] = (int8_t)sd;
    // first layer: add site d; units of degree d become final
#pragma unroll
    for (int j = 0; j < HPL; ++j) {
      const int k = lane + 32 * j;
      const int m = made_degree(k, N);
      if (m >= d) a[j] = fmaf(D.W1t[(int64_t)(d - 1) * H + k], sd, a[j]);
      if (m == d) h1[k] = fmaxf(a[j], 0.f);
    }
    __syncwarp();
    // second layer: units of degree d (k2 = d-1, d-1 + (N-1), ...) become computable
    for (int k2 = d - 1; k2 < H; k2 += N - 1) {
      float part = 0.f;
#pragma unroll
      for (int j = 0; j < HPL; ++j) {
        const int k1 = lane + 32 * j;
        if (made_degree(k1, N) <= d) part = fmaf(D.W2[(int64_t)k2 * H + k1], h1[k1], part);
      }
      const float a2 = warp_sum(part) + D.b2[k2];
      if (lane == 0) h2[k2] = fmaxf(a2, 0.f);
    }
    __syncwarp();
  }
  for (int i = lane; i < N; i += 32) spins[c * N + i] = s[i];
  if (lane == 0 && logq) logq[c] = lq;
}

// ---------------------------------------------------------------------------------------
// Independent Metropolis-Hastings: chain c takes the proposal (its own draw from q) iff
//   ln u < 2 Re[log psi(s') - log psi(s)] + log q(s) - log q(s'),
//   u from Philox4x64-10({c, round, 0, 3}, {seed, stream}) word 1 as in the local moves.
// One warp per chain (the warp copies the accepted configuration).
// ---------------------------------------------------------------------------------------
__global__ void k_made_mh(int64_t C, int N, const int8_t* __restrict__ prop,
                          const float2* __restrict__ prop_lp, const float* __restrict__ prop_lq,
                          int8_t* __restrict__ chains, float2* __restrict__ chain_lp,
                          float* __restrict__ chain_lq, uint64_t seed, uint64_t stream,
                          uint64_t round, unsigned long long* accepts) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= C) return;
  const u64x4 w = philox4x64_10((uint64_t)c, round, 0ull, 3ull, seed, stream);
  const float u = ((float)(uint32_t)(w.w1 >> 40) + 0.5f) * 5.9604644775390625e-08f;
  const float delta = 2.f * (prop_lp[c].x - chain_lp[c].x) + chain_lq[c] - prop_lq[c];
  const bool acc = logf(u) < delta;
  if (acc) {
    for (int i = lane; i < N; i += 32) chains[c * N + i] = prop[c * N + i];
    if (lane == 0) {
      chain_lp[c] = prop_lp[c];
      chain_lq[c] = prop_lq[c];
      atomicAdd(accepts, 1ull);
    }
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
#define MADE_DISPATCH(H, ...)                                       \
  switch ((H) / 32) {                                               \
    case 1: { constexpr int HPL = 1; __VA_ARGS__; } break;          \
    case 2: { constexpr int HPL = 2; __VA_ARGS__; } break;          \
    case 4: { constexpr int HPL = 4; __VA_ARGS__; } break;          \
    case 8: { constexpr int HPL = 8; __VA_ARGS__; } break;          \
    case 16: { constexpr int HPL = 16; __VA_ARGS__; } break;        \
    default: return cudaErrorInvalidValue;                          \
  }

static size_t made_smem(int N, int H) {
  return (size_t)4 * (2 * H * sizeof(float)) + (size_t)4 * ((N + 15) & ~15);
}

cudaError_t launch_made_transpose(const MadeDev& D, cudaStream_t st) {
  const int64_t tot = 2 * (int64_t)D.H * D.N + (int64_t)D.H * D.H;
  k_made_transpose<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, st>>>(D);
  return cudaGetLastError();
}

cudaError_t launch_made_logq(const MadeDev& D, const int8_t* spins, int64_t n, float* logq,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 3) / 4);
  MADE_DISPATCH(D.H, k_made_fwd<HPL><<<grid, 128, made_smem(D.N, D.H), st>>>(
                         D, spins, n, logq, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f));
  return cudaGetLastError();
}

cudaError_t launch_made_grad(const MadeDev& D, const int8_t* spins, int64_t n, MadeWork& w,
                             float* grad, cudaStream_t st) {
  const int N = D.N, H = D.H;
  const unsigned grid = (unsigned)((n + 3) / 4);
  MADE_DISPATCH(H, k_made_fwd<HPL><<<grid, 128, made_smem(N, H), st>>>(
                       D, spins, n, w.logq, w.H1, w.H2, w.G1, w.G2, w.G3, 1.f / (float)n));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float* gW1 = grad;
  float* gb1 = gW1 + (int64_t)H * N;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (int64_t)H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + (int64_t)N * H;
  k_made_outer<1><<<dim3((N + 63) / 64, (H + 63) / 64), 256, 0, st>>>(w.G1, spins, n, H, N, N, gW1);
  k_made_outer<2><<<dim3((H + 63) / 64, (H + 63) / 64), 256, 0, st>>>(w.G2, w.H1, n, H, H, N, gW2);
  k_made_outer<3><<<dim3((H + 63) / 64, (N + 63) / 64), 256, 0, st>>>(w.G3, w.H2, n, N, H, N, gW3);
  k_made_colsum<<<(H + 127) / 128, 128, 0, st>>>(w.G1, n, H, gb1);
  k_made_colsum<<<(H + 127) / 128, 128, 0, st>>>(w.G2, n, H, gb2);
  k_made_colsum<<<(N + 127) / 128, 128, 0, st>>>(w.G3, n, N, gb3);
  return cudaGetLastError();
}

cudaError_t launch_made_fwd_bwd(const MadeDev& D, const int8_t* spins, int64_t n, MadeWork& w,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 3) / 4);
  MADE_DISPATCH(D.H, k_made_fwd<HPL><<<grid, 128, made_smem(D.N, D.H), st>>>(
                         D, spins, n, w.logq, w.H1, w.H2, w.G1, w.G2, w.G3, 1.f));
  return cudaGetLastError();
}

cudaError_t launch_adam(float* th, float* m, float* v, const float* g, int64_t np, int t, float lr,
                        cudaStream_t st) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)t)));
  const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)t)));
  k_adam<<<(unsigned)std::min<int64_t>((np + 255) / 256, 4096), 256, 0, st>>>(
      th, m, v, g, np, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_made_sample(const MadeDev& D, int64_t n, uint64_t seed, uint64_t stream,
                               uint64_t round, int8_t* spins, float* logq, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 3) / 4);
  MADE_DISPATCH(D.H, k_made_sample<HPL><<<grid, 128, made_smem(D.N, D.H), st>>>(
                         D, n, seed, stream, round, spins, logq));
  return cudaGetLastError();
}

cudaError_t launch_made_mh(int64_t C, int N, const int8_t* prop, const float2* prop_lp,
                           const float* prop_lq, int8_t* chains, float2* chain_lp,
                           float* chain_lq, uint64_t seed, uint64_t stream, uint64_t round,
                           unsigned long long* accepts, cudaStream_t st) {
  k_made_mh<<<(unsigned)((C + 3) / 4), 128, 0, st>>>(C, N, prop, prop_lp, prop_lq, chains, chain_lp,
                                                    chain_lq, seed, stream, round, accepts);
  return cudaGetLastError();
}

}  // namespace vmc
