// rbm.cu -- complex-RBM evaluation kernels of the VMC step: parameter preparation, log psi,
// the fused local energy, theta/tanh theta and the dense log-derivatives.
#include "rbm_warp.cuh"

namespace vmc {

// ---------------------------------------------------------------------------------------
// a1: FP64 master parameters -> FP32 working copies.  Wt is W transposed ([N][M]) so that
// the column W[:, i] a proposal needs is contiguous across the warp's lanes.
// ---------------------------------------------------------------------------------------
__global__ void k_param_prep(const double2* __restrict__ p, int N, int M, float2* __restrict__ a,
                             float2* __restrict__ b, float2* __restrict__ Wt) {
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    double2 v = p[k];
    float2 f = make_float2((float)v.x, (float)v.y);
    if (k < N) a[k] = f;
    else if (k < N + M) b[k - N] = f;
    else {
      int64_t q = k - N - M;
      int j = (int)(q / N), i = (int)(q % N);
      Wt[(int64_t)i * M + j] = f;
    }
  }
}

// Move tables (see RbmDev), one block per move: D from the FP64 W, tanh D and log cosh D in
// FP64, the tanh rounded once to FP32 and the log cosh summed over k in FP64 first; the
// prefactors exp(sum_k log cosh D_qk - da) for both spins of the move's first site from
// that FP64 sum and the FP64 visible biases.
//   log cosh z = z' - ln 2 + log(1 + exp(-2 z')),  z' = z or -z with Re z' >= 0,
// which stays finite for any |Re D|.
__global__ void __launch_bounds__(128) k_move_tables(const double2* __restrict__ p, int N, int M,
                                                     int model, int Lx, int Ly,
                                                     float2* __restrict__ mth,
                                                     float2* __restrict__ mlc,
                                                     float2* __restrict__ mpre) {
  const int q = blockIdx.x;
  const double2* W = p + N + M;                  // W[k][i] at k * N + i
  int i = q, j = -1;
  if (model == 1) bond_ends(Lx, Ly, q, &i, &j);
  double lre = 0.0, lim = 0.0;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const double2 wi = W[(int64_t)k * N + i];
    double dx = 2.0 * wi.x, dy = 2.0 * wi.y;
    if (j >= 0) {
      const double2 wj = W[(int64_t)k * N + j];
      dx -= 2.0 * wj.x;
      dy -= 2.0 * wj.y;
    }
    double sy, cy;
    sincos(dy, &sy, &cy);
    const double chx = cosh(dx), shx = sinh(dx);
    const double cr = chx * cy, ci = shx * sy;   // cosh(dx + i dy)
    const double sr = shx * cy, si = chx * sy;   // sinh(dx + i dy)
    const double den = cr * cr + ci * ci;
    mth[(int64_t)q * M + k] =
        make_float2((float)((sr * cr + si * ci) / den), (float)((si * cr - sr * ci) / den));
    const double zx = dx >= 0.0 ? dx : -dx, zy = dx >= 0.0 ? dy : -dy;
    const double e = exp(-2.0 * zx);
    double s2, c2;
    sincos(-2.0 * zy, &s2, &c2);
    const double wr = 1.0 + e * c2, wim = e * s2;
    lre += zx - 0.69314718055994530942 + 0.5 * log(wr * wr + wim * wim);
    lim += zy + atan2(wim, wr);
  }
  __shared__ double red[2][4];
  for (int o = 16; o > 0; o >>= 1) {
    lre += __shfl_xor_sync(0xffffffffu, lre, o);
    lim += __shfl_xor_sync(0xffffffffu, lim, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = lre;
    red[1][threadIdx.x >> 5] = lim;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double re = red[0][0] + red[0][1] + red[0][2] + red[0][3];
    const double im = red[1][0] + red[1][1] + red[1][2] + red[1][3];
    const double twopi = 6.28318530717958647692;
    mlc[q] = make_float2((float)re, (float)(im - twopi * rint(im / twopi)));
    double2 da = p[i];                            // a_i (- a_j): the visible-bias difference
    if (j >= 0) {
      da.x -= p[j].x;
      da.y -= p[j].y;
    }
    for (int h = 0; h < 2; ++h) {
      const double s2 = h ? -2.0 : 2.0;
      const double lx = re - s2 * da.x, ly = im - s2 * da.y;
      const double mag = exp(lx);
      mpre[2 * q + h] = make_float2((float)(mag * cos(ly)), (float)(mag * sin(ly)));
    }
  }
}

cudaError_t launch_move_tables(const double2* p, int N, int M, int model, int Lx, int Ly,
                               float2* mth, float2* mlc, float2* mpre, cudaStream_t st) {
  const int moves = model == 1 ? num_bonds(Lx, Ly) : N;
  k_move_tables<<<moves, 128, 0, st>>>(p, N, M, model, Lx, Ly, mth, mlc, mpre);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// batch kernels: one warp per configuration
// ---------------------------------------------------------------------------------------
template <int MPL>
__global__ void __launch_bounds__(128) k_logpsi(RbmDev R, const int8_t* __restrict__ spins,
                                                int64_t n, float2* __restrict__ out,
                                                unsigned* status) {
  extern __shared__ int8_t sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (q >= n) return;
  const int Npad = (R.N + 15) & ~15;
  int8_t* s = sm + wib * Npad;
  for (int i = lane; i < R.N; i += 32) s[i] = spins[q * R.N + i];
  __syncwarp();
  float2 th[MPL];
  warp_theta<MPL>(R, s, lane, th);
  float2 lp = warp_logpsi<MPL>(R, s, lane, th);
  if (lane == 0) {
    out[q] = lp;
    if (!isfinite(lp.x) || !isfinite(lp.y)) flag_error(status, DEV_ERR_NUMERIC);
  }
}

template <int MPL>
__global__ void __launch_bounds__(128) k_eloc(RbmDev R, LatDev L,
                                              const int8_t* __restrict__ spins, int64_t n,
                                              float2* __restrict__ out, unsigned* status) {
  extern __shared__ int8_t sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (q >= n) return;
  const int Npad = (R.N + 15) & ~15;
  int8_t* s = sm + wib * Npad;
  for (int i = lane; i < R.N; i += 32) s[i] = spins[q * R.N + i];
  __syncwarp();
  float2 th[MPL], t[MPL];
  warp_theta<MPL>(R, s, lane, th);
#pragma unroll
  for (int k = 0; k < MPL; ++k) t[k] = tanh_c(th[k].x, th[k].y);
  float2 e = warp_eloc<MPL>(R, L, s, lane, t, eloc_buffer(sm, R.N, wib));
  if (lane == 0) {
    out[q] = e;
    if (!isfinite(e.x) || !isfinite(e.y)) flag_error(status, DEV_ERR_NUMERIC);
  }
}

// tanh theta for a batch: T[n][M] (the b- and W-block log-derivative factors)
template <int MPL>
__global__ void __launch_bounds__(128) k_theta_tanh(RbmDev R, const int8_t* __restrict__ spins,
                                                    int64_t n, float2* __restrict__ T) {
  extern __shared__ int8_t sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (q >= n) return;
  const int Npad = (R.N + 15) & ~15;
  int8_t* s = sm + wib * Npad;
  for (int i = lane; i < R.N; i += 32) s[i] = spins[q * R.N + i];
  __syncwarp();
  float2 th[MPL];
  warp_theta<MPL>(R, s, lane, th);
#pragma unroll
  for (int k = 0; k < MPL; ++k) {
    int hj = lane + 32 * k;
    if (hj < R.M) T[q * R.M + hj] = tanh_c(th[k].x, th[k].y);
  }
}

// dense log-derivatives O[n][P] = [s | t | t (x) s] (FP32 complex)
__global__ void k_ok_dense(const int8_t* __restrict__ spins, const float2* __restrict__ T,
                           int64_t n, int N, int M, float2* __restrict__ O) {
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  const int64_t total = n * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = e / P, k = e % P;
    float2 v;
    if (k < N) v = make_float2((float)spins[q * N + k], 0.f);
    else if (k < N + M) v = T[q * M + (k - N)];
    else {
      int64_t r = k - N - M;
      int j = (int)(r / N), i = (int)(r % N);
      float si = (float)spins[q * N + i];
      float2 t = T[q * M + j];
      v = make_float2(si * t.x, si * t.y);
    }
    O[e] = v;
  }
}

// theta for a batch of configurations: 64 configurations x 64 hidden units per block,
// K (the sites) in slices of 32 through shared memory; thread (tq, tj) owns configurations
// tq + 16 a and units tj + 16 b (a, b < 4) and runs each entry's chain of fused
// multiply-adds over i in increasing order, starting from b_j.
constexpr int TG_Q = 64, TG_J = 64, TG_K = 32;
__global__ void __launch_bounds__(256) k_theta_gemm(const float2* __restrict__ b,
                                                    const float2* __restrict__ Wt, int N, int M,
                                                    const int8_t* __restrict__ spins, int64_t C,
                                                    float2* __restrict__ theta) {
  __shared__ float2 Ws[TG_K][TG_J + 1];
  __shared__ float Ss[TG_Q][TG_K + 1];
  const int tid = threadIdx.x, tq = tid & 15, tj = tid >> 4;
  const int64_t q0 = (int64_t)blockIdx.x * TG_Q;
  const int j0 = blockIdx.y * TG_J;
  float2 acc[4][4];
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    const int j = j0 + tj + 16 * bb;
    const float2 bj = (j < M) ? b[j] : make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a][bb] = bj;
  }
  for (int k0 = 0; k0 < N; k0 += TG_K) {
    for (int e = tid; e < TG_K * TG_J; e += 256) {
      const int kk = e / TG_J, jj = e % TG_J;
      const int i = k0 + kk, j = j0 + jj;
      Ws[kk][jj] = (i < N && j < M) ? Wt[(int64_t)i * M + j] : make_float2(0.f, 0.f);
    }
    for (int e = tid; e < TG_Q * TG_K; e += 256) {
      const int qq = e / TG_K, kk = e % TG_K;
      const int64_t q = q0 + qq;
      const int i = k0 + kk;
      Ss[qq][kk] = (q < C && i < N) ? (float)spins[q * N + i] : 0.f;
    }
    __syncthreads();
    const int kn = min(TG_K, N - k0);
    for (int kk = 0; kk < kn; ++kk) {
      float sv[4];
      float2 wv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) sv[a] = Ss[tq + 16 * a][kk];
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) wv[bb] = Ws[kk][tj + 16 * bb];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          acc[a][bb].x = fmaf(sv[a], wv[bb].x, acc[a][bb].x);
          acc[a][bb].y = fmaf(sv[a], wv[bb].y, acc[a][bb].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t q = q0 + tq + 16 * a;
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const int j = j0 + tj + 16 * bb;
      if (q < C && j < M) theta[q * M + j] = acc[a][bb];
    }
  }
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
cudaError_t launch_param_prep(const double2* p, int N, int M, float2* a, float2* b, float2* Wt,
                              cudaStream_t st) {
  int64_t P = (int64_t)N + M + (int64_t)N * M;
  int blocks = (int)std::min<int64_t>((P + 255) / 256, 4096);
  k_param_prep<<<blocks, 256, 0, st>>>(p, N, M, a, b, Wt);
  return cudaGetLastError();
}

cudaError_t launch_logpsi(const RbmDev& R, const int8_t* spins, int64_t n, float2* out,
                          unsigned* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  unsigned grid = (unsigned)((n + kWarps - 1) / kWarps);
  VMC_DISPATCH_MPL(R.M, k_logpsi<MPL><<<grid, 32 * kWarps, spin_smem(R.N), st>>>(R, spins, n, out, status));
  return cudaGetLastError();
}

cudaError_t launch_eloc(const RbmDev& R, const LatDev& L, const int8_t* spins, int64_t n,
                        float2* out, unsigned* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  unsigned grid = (unsigned)((n + kWarps - 1) / kWarps);
  VMC_DISPATCH_MPL(R.M, k_eloc<MPL><<<grid, 32 * kWarps, sample_smem(R.N), st>>>(R, L, spins, n, out, status));
  return cudaGetLastError();
}

cudaError_t launch_theta_tanh(const RbmDev& R, const int8_t* spins, int64_t n, float2* T,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  unsigned grid = (unsigned)((n + kWarps - 1) / kWarps);
  VMC_DISPATCH_MPL(R.M, k_theta_tanh<MPL><<<grid, 32 * kWarps, spin_smem(R.N), st>>>(R, spins, n, T));
  return cudaGetLastError();
}

cudaError_t launch_theta_gemm(const RbmDev& R, const int8_t* spins, int64_t C, float2* theta,
                              cudaStream_t st) {
  if (C <= 0) return cudaSuccess;
  dim3 grid((unsigned)((C + TG_Q - 1) / TG_Q), (unsigned)((R.M + TG_J - 1) / TG_J));
  k_theta_gemm<<<grid, 256, 0, st>>>(R.b, R.Wt, R.N, R.M, spins, C, theta);
  return cudaGetLastError();
}

cudaError_t launch_ok_dense(const int8_t* spins, const float2* T, int64_t n, int N, int M,
                            float2* O, cudaStream_t st) {
  int64_t P = (int64_t)N + M + (int64_t)N * M;
  int64_t total = n * P;
  if (total <= 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 65536);
  k_ok_dense<<<blocks, 256, 0, st>>>(spins, T, n, N, M, O);
  return cudaGetLastError();
}

}  // namespace vmc
