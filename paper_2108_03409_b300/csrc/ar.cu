// ar.cu -- the autoregressive network as the variational ansatz (arXiv:2108.03409, section
// "Autoregressive neural quantum states"): psi(s) = q(s)^(1/2) with q the masked
// autoregressive network of made.cu (normalised, sum_s q(s) = 1), so samples are exact
// independent draws (k_made_sample) instead of a Markov chain.  Real parameters and real,
// positive amplitudes (the TFIM's ground state is positive); the SR equation is real:
//   O_k(s) = (1/2) d log q(s) / d theta_k = -(1/2) d(-log q(s)) / d theta_k,
//   E_loc(s) = sum_s' H_ss' (q(s') / q(s))^(1/2).
// The per-sample gradients of -log q come from the network's backward pass (G1, G2, G3 at
// the units, H1, H2 the activations), and O_k is formed from them on the fly:
//   W1[k][d]: G1_k s_d (m(k) >= d+1),  b1[k]: G1_k,  W2[k2][k1]: G2_k2 H1_k1 (m(k2) >= m(k1)),
//   b2[k2]: G2_k2,  W3[d][k2]: G3_d H2_k2 (d+1 > m(k2)),  b3[d]: G3_d;  masked entries 0.
#include <cmath>

#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

namespace {

__device__ __forceinline__ int ar_degree(int k, int N) { return (k % (N - 1)) + 1; }

// the per-sample derivative of -log q(s) with respect to parameter k (canonical layout)
__device__ __forceinline__ float ar_dl(const int8_t* __restrict__ s, const float* __restrict__ g1,
                                       const float* __restrict__ g2, const float* __restrict__ g3,
                                       const float* __restrict__ h1, const float* __restrict__ h2,
                                       int N, int H, int64_t k) {
  const int64_t nW1 = (int64_t)H * N, nW2 = (int64_t)H * H, nW3 = (int64_t)N * H;
  if (k < nW1) {
    const int kk = (int)(k / N), d = (int)(k % N);
    return ar_degree(kk, N) >= d + 1 ? g1[kk] * (float)s[d] : 0.f;
  }
  k -= nW1;
  if (k < H) return g1[k];
  k -= H;
  if (k < nW2) {
    const int k2 = (int)(k / H), k1 = (int)(k % H);
    return ar_degree(k2, N) >= ar_degree(k1, N) ? g2[k2] * h1[k1] : 0.f;
  }
  k -= nW2;
  if (k < H) return g2[k];
  k -= H;
  if (k < nW3) {
    const int d = (int)(k / H), k2 = (int)(k % H);
    return d + 1 > ar_degree(k2, N) ? g3[d] * h2[k2] : 0.f;
  }
  k -= nW3;
  return g3[k];
}

__global__ void k_ar_connected(const int8_t* __restrict__ spins, int64_t n, LatDev L, int K,
                               int8_t* __restrict__ out) {
  const int N = L.Lx * L.Ly;
  const int64_t tot = n * K * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / ((int64_t)K * N);
    const int r = (int)(e % ((int64_t)K * N));
    const int k = r / N, i = r % N;
    const int8_t* s = spins + q * N;
    int8_t v = s[i];
    if (L.model == 0) {
      if (i == k) v = -v;                         // flip site k
    } else {
      int a, b;
      bond_ends(L.Lx, L.Ly, k, &a, &b);
      if (s[a] != s[b] && (i == a || i == b)) v = -v;   // exchange an anti-parallel pair
    }
    out[e] = v;
  }
}

__global__ void k_ar_eloc(const int8_t* __restrict__ spins, const float* __restrict__ lq,
                          const float* __restrict__ lqc, int64_t n, LatDev L, int K,
                          float2* __restrict__ E, unsigned* status) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int N = L.Lx * L.Ly;
  const int8_t* s = spins + q * N;
  float zz = 0.f;
  for (int b = 0; b < L.nb; ++b) {
    int i, j;
    bond_ends(L.Lx, L.Ly, b, &i, &j);
    zz += (float)(s[i] * s[j]);
  }
  const float l0 = lq[q];
  float e;
  if (L.model == 0) {
    e = -L.J * zz;
    for (int k = 0; k < K; ++k) e = fmaf(-L.h, expf(0.5f * (lqc[q * K + k] - l0)), e);
  } else {
    e = L.J * zz;
    for (int k = 0; k < K; ++k) {
      int i, j;
      bond_ends(L.Lx, L.Ly, k, &i, &j);
      if (s[i] != s[j]) e = fmaf(2.f * L.J, expf(0.5f * (lqc[q * K + k] - l0)), e);
    }
  }
  if (!isfinite(e)) flag_error(status, DEV_ERR_NUMERIC);
  E[q] = make_float2(e, 0.f);
}

// thread per parameter, blockIdx.y a chunk of samples; part[chunk][k] = {sum O, sum O (E-<E>)}
__global__ void k_ar_moments(const int8_t* __restrict__ spins, const float* __restrict__ G1,
                             const float* __restrict__ G2, const float* __restrict__ G3,
                             const float* __restrict__ H1, const float* __restrict__ H2,
                             const float2* __restrict__ E, const double* __restrict__ estats,
                             int64_t n, int N, int H, int64_t P, int64_t chunk,
                             double2* __restrict__ part) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const int64_t q0 = (int64_t)blockIdx.y * chunk, q1 = min(n, q0 + chunk);
  const double em = estats[0];
  double so = 0.0, sf = 0.0;
  for (int64_t q = q0; q < q1; ++q) {
    const double o = -0.5 * (double)ar_dl(spins + q * N, G1 + q * H, G2 + q * H, G3 + q * N,
                                          H1 + q * H, H2 + q * H, N, H, k);
    so += o;
    sf = fma(o, (double)E[q].x - em, sf);
  }
  part[(int64_t)blockIdx.y * P + k] = make_double2(so, sf);
}

__global__ void k_ar_moments_reduce(const double2* __restrict__ part, int chunks, int64_t P,
                                    double inv_n, double2* meanO, double2* F) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  double so = 0.0, sf = 0.0;
  for (int c = 0; c < chunks; ++c) {
    const double2 v = part[(int64_t)c * P + k];
    so += v.x;
    sf += v.y;
  }
  meanO[k] = make_double2(so * inv_n, 0.0);
  F[k] = make_double2(sf * inv_n, 0.0);
}

// X[k][q] = O_k(q) - <O_k> (the Gram's real-row mode); zero beyond n and beyond P
__global__ void k_ar_build_x(const int8_t* __restrict__ spins, const float* __restrict__ G1,
                             const float* __restrict__ G2, const float* __restrict__ G3,
                             const float* __restrict__ H1, const float* __restrict__ H2,
                             const double2* __restrict__ meanO, int64_t n, int N, int H,
                             int64_t P, int64_t rows_pad, int64_t ld, float* __restrict__ X) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t k = blockIdx.y;
  if (q >= ld) return;
  float v = 0.f;
  if (k < P && q < n)
    v = (float)(-0.5 * (double)ar_dl(spins + q * N, G1 + q * H, G2 + q * H, G3 + q * N,
                                     H1 + q * H, H2 + q * H, N, H, k) - meanO[k].x);
  X[k * ld + q] = v;
}

__global__ void k_freeze_zero_rows(double2* S, double2* F, int64_t P) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  if (S[k * P + k].x == 0.0) {
    S[k * P + k] = make_double2(1.0, 0.0);
    F[k] = make_double2(0.0, 0.0);
  }
}

__global__ void k_ar_update(double* theta, const double2* x, int64_t P, double dt, float* t32) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const double v = theta[k] - dt * x[k].x;
  theta[k] = v;
  t32[k] = (float)v;
}

__global__ void k_to_f32_real(const double* a, int64_t n, float* b) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) b[k] = (float)a[k];
}

__global__ void k_scale_f32(float* x, int64_t n, float a) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) x[k] *= a;
}

// dense per-sample O [n][P]
__global__ void k_ar_dense_o(const int8_t* __restrict__ spins, const float* __restrict__ G1,
                             const float* __restrict__ G2, const float* __restrict__ G3,
                             const float* __restrict__ H1, const float* __restrict__ H2, int64_t n,
                             int N, int H, int64_t P, float* __restrict__ O) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * P) return;
  const int64_t q = e / P, k = e % P;
  O[e] = -0.5f * ar_dl(spins + q * N, G1 + q * H, G2 + q * H, G3 + q * N, H1 + q * H, H2 + q * H,
                       N, H, k);
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_ar_connected(const int8_t* spins, int64_t n, const LatDev& L, int8_t* out,
                                cudaStream_t st) {
  const int N = L.Lx * L.Ly;
  const int K = L.model == 0 ? N : L.nb;
  const int64_t tot = n * K * N;
  k_ar_connected<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 1 << 20), 256, 0, st>>>(
      spins, n, L, K, out);
  return cudaGetLastError();
}

cudaError_t launch_ar_eloc(const int8_t* spins, const float* lq, const float* lq_conn, int64_t n,
                           const LatDev& L, float2* E, unsigned* status, cudaStream_t st) {
  const int K = L.model == 0 ? L.Lx * L.Ly : L.nb;
  k_ar_eloc<<<blocks_for(n), 256, 0, st>>>(spins, lq, lq_conn, n, L, K, E, status);
  return cudaGetLastError();
}

cudaError_t launch_ar_moments(const int8_t* spins, const MadeWork& w, const float2* E,
                              const double* estats, int64_t n, int N, int H, double* part,
                              int64_t part_cap, double2* meanO, double2* F, cudaStream_t st) {
  const int64_t P = made_nparams(N, H);
  const int64_t kb = (P + 255) / 256;
  int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((4 * 148 + kb - 1) / kb, n / 256));
  chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, part_cap / (2 * P)));
  const int64_t chunk = (n + chunks - 1) / chunks;
  chunks = (n + chunk - 1) / chunk;
  double2* p2 = reinterpret_cast<double2*>(part);
  k_ar_moments<<<dim3((unsigned)kb, (unsigned)chunks), 256, 0, st>>>(
      spins, w.G1, w.G2, w.G3, w.H1, w.H2, E, estats, n, N, H, P, chunk, p2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ar_moments_reduce<<<(unsigned)kb, 256, 0, st>>>(p2, (int)chunks, P, 1.0 / (double)n, meanO, F);
  return cudaGetLastError();
}

cudaError_t launch_ar_build_x(const int8_t* spins, const MadeWork& w, const double2* meanO,
                              int64_t n, int N, int H, int64_t rows_pad, int64_t ld, float* X,
                              cudaStream_t st) {
  const int64_t P = made_nparams(N, H);
  if (P > rows_pad || n > ld || rows_pad > 65535) return cudaErrorInvalidValue;
  k_ar_build_x<<<dim3(blocks_for(ld), (unsigned)rows_pad), 256, 0, st>>>(
      spins, w.G1, w.G2, w.G3, w.H1, w.H2, meanO, n, N, H, P, rows_pad, ld, X);
  return cudaGetLastError();
}

cudaError_t launch_freeze_zero_rows(double2* S, double2* F, int64_t P, cudaStream_t st) {
  k_freeze_zero_rows<<<blocks_for(P), 256, 0, st>>>(S, F, P);
  return cudaGetLastError();
}

cudaError_t launch_ar_update(double* theta, const double2* x, int64_t P, double dt, float* theta32,
                             cudaStream_t st) {
  k_ar_update<<<blocks_for(P), 256, 0, st>>>(theta, x, P, dt, theta32);
  return cudaGetLastError();
}

cudaError_t launch_scale_f32(float* x, int64_t n, float a, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_scale_f32<<<blocks_for(n), 256, 0, st>>>(x, n, a);
  return cudaGetLastError();
}

cudaError_t launch_ar_dense_o(const int8_t* spins, const MadeWork& w, int64_t n, int N, int H,
                              float* O, cudaStream_t st) {
  const int64_t P = made_nparams(N, H);
  k_ar_dense_o<<<blocks_for(n * P), 256, 0, st>>>(spins, w.G1, w.G2, w.G3, w.H1, w.H2, n, N, H, P, O);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* a, int64_t n, float* b, cudaStream_t st) {
  k_to_f32_real<<<blocks_for(n), 256, 0, st>>>(a, n, b);
  return cudaGetLastError();
}

}  // namespace vmc
