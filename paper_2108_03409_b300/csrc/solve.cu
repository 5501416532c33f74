// solve.cu -- regularised solve of S~ x = F (section "Diagonal shift"; Algorithm 1,
// solve_TDVP_equation) by a blocked right-looking complex Cholesky factorisation
// S~ = L L^H, in FP64, or in FP32 followed by FP64 iterative refinement against the
// FP64 S~.  Diagonal blocks of L are inverted once so that the panel solve and the
// triangular solves become small matrix products.
#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

static constexpr int NB = 64;

template <typename C> struct RealOf;
template <> struct RealOf<double2> { typedef double T; };
template <> struct RealOf<float2> { typedef float T; };

template <typename C> __device__ __forceinline__ C mk(double x, double y) {
  typedef typename RealOf<C>::T R;
  C c;
  c.x = (R)x;
  c.y = (R)y;
  return c;
}
template <typename C> __device__ __forceinline__ C cmul_t(C a, C b) {
  C c;
  c.x = a.x * b.x - a.y * b.y;
  c.y = a.x * b.y + a.y * b.x;
  return c;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc_t(C a, C b) {
  C c;
  c.x = a.x * b.x + a.y * b.y;
  c.y = a.y * b.x - a.x * b.y;
  return c;
}
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {  // acc += a*b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
template <typename C> __device__ __forceinline__ void cfmac(C& acc, C a, C b) {  // acc += a*conj(b)
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y);
  acc.y = fma(-a.x, b.y, acc.y);
}

// A = S (+ shift on the diagonal), converted to the factor's precision
template <typename C>
__global__ void k_copy_shift(const double2* __restrict__ S, C* __restrict__ A, int64_t P,
                             double nu, int mode) {
  const int64_t total = P * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 v = S[e];
    const int64_t r = e / P, c = e % P;
    if (r == c) v.x = (mode == 0) ? v.x * (1.0 + nu) : v.x + nu;
    A[e] = mk<C>(v.x, v.y);
  }
}

// Factor the diagonal block (rows/cols k0..k0+kw) in shared memory and store its inverse.
// 256 threads: column c is scaled, then the trailing lower triangle (r, cc), c < cc <= r,
// is updated with all threads striding over it; the inverse is built row by row
// (Linv[rr][c] = -sum_{m=c}^{rr-1} L[rr][m] Linv[m][c] / L[rr][rr]) with four threads per
// column sharing the sum.
constexpr int POTRF_THREADS = 256;

template <typename C>
__global__ void __launch_bounds__(POTRF_THREADS) k_potrf_diag(C* __restrict__ A, int64_t P,
                                                              int64_t k0, int kw,
                                                              C* __restrict__ Dinv,
                                                              unsigned* status) {
  typedef typename RealOf<C>::T R;
  extern __shared__ unsigned char psm[];
  C* a = reinterpret_cast<C*>(psm);           // [NB][NB+1]
  C* inv = a + NB * (NB + 1);                 // [NB][NB+1]
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += POTRF_THREADS) {
    const int r = e / NB, c = e % NB;
    a[r * (NB + 1) + c] = (r < kw && c <= r) ? A[(k0 + r) * P + k0 + c] : mk<C>(0.0, 0.0);
    inv[r * (NB + 1) + c] = mk<C>(0.0, 0.0);
  }
  __syncthreads();
  bool bad = false;
  for (int c = 0; c < kw; ++c) {
    R d = a[c * (NB + 1) + c].x;
    if (!(d > (R)0) || !isfinite(d)) { bad = true; d = (R)1; }
    const R lcc = sqrt(d);
    const R ilcc = (R)1 / lcc;
    __syncthreads();                          // everyone has read the pivot
    for (int r = c + 1 + tid; r < kw; r += POTRF_THREADS) {
      C v = a[r * (NB + 1) + c];
      v.x *= ilcc;
      v.y *= ilcc;
      a[r * (NB + 1) + c] = v;
    }
    if (tid == 0) a[c * (NB + 1) + c] = mk<C>((double)lcc, 0.0);
    __syncthreads();
    const int m = kw - c - 1;
    for (int e = tid; e < m * m; e += POTRF_THREADS) {
      const int rr = c + 1 + e / m, cc = c + 1 + e % m;
      if (cc > rr) continue;
      const C lr = a[rr * (NB + 1) + c], lc = a[cc * (NB + 1) + c];
      C v = a[rr * (NB + 1) + cc];
      v.x -= lr.x * lc.x + lr.y * lc.y;       // v -= l_rc * conj(l_cc,c)
      v.y -= lr.y * lc.x - lr.x * lc.y;
      a[rr * (NB + 1) + cc] = v;
    }
    __syncthreads();
  }
  if (bad && tid == 0) flag_error(status, DEV_ERR_NUMERIC);
  for (int e = tid; e < kw * kw; e += POTRF_THREADS) {
    const int r = e / kw, c = e % kw;
    if (c <= r) A[(k0 + r) * P + k0 + c] = a[r * (NB + 1) + c];
  }
  // inverse of the lower-triangular block, row by row
  if (tid < kw) inv[tid * (NB + 1) + tid] = mk<C>(1.0 / (double)a[tid * (NB + 1) + tid].x, 0.0);
  __syncthreads();
  const int col = tid >> 2, part = tid & 3;
  for (int rr = 1; rr < kw; ++rr) {
    C s = mk<C>(0.0, 0.0);
    if (col < rr)
      for (int mm = col + part; mm < rr; mm += 4) cfma(s, a[rr * (NB + 1) + mm], inv[mm * (NB + 1) + col]);
    s.x += __shfl_xor_sync(0xffffffffu, s.x, 1);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, 1);
    s.x += __shfl_xor_sync(0xffffffffu, s.x, 2);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, 2);
    if (col < rr && part == 0) {
      const R lrr = a[rr * (NB + 1) + rr].x;
      inv[rr * (NB + 1) + col] = mk<C>(-(double)s.x / (double)lrr, -(double)s.y / (double)lrr);
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += POTRF_THREADS) {
    const int r = e / NB, c = e % NB;
    Dinv[e] = (r < kw && c < kw) ? inv[r * (NB + 1) + c] : mk<C>(0.0, 0.0);
  }
}

// Panel: X = B L_kk^{-H}, X[r][c] = sum_{m<=c} B[r][m] conj(Linv[c][m]) for the rows
// below the diagonal block; 64 rows per block, written over the panel of A.
template <typename C>
__global__ void __launch_bounds__(256) k_trsm_inv(C* __restrict__ A, int64_t P, int64_t k0,
                                                  int kw, const C* __restrict__ Dinv) {
  extern __shared__ unsigned char tsm[];
  C* B = reinterpret_cast<C*>(tsm);            // [NB][NB+1]
  C* Li = B + NB * (NB + 1);                   // [NB][NB+1]
  const int64_t r0 = k0 + kw + (int64_t)blockIdx.x * NB;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += 256) {
    const int rr = e / NB, c = e % NB;
    Li[rr * (NB + 1) + c] = Dinv[e];
    const int64_t row = r0 + rr;
    B[rr * (NB + 1) + c] = (row < P && c < kw) ? A[row * P + k0 + c] : mk<C>(0.0, 0.0);
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += 256) {
    const int rr = e / NB, c = e % NB;
    const int64_t row = r0 + rr;
    if (row >= P || c >= kw) continue;
    C s = mk<C>(0.0, 0.0);
    for (int m = 0; m <= c; ++m) cfmac(s, B[rr * (NB + 1) + m], Li[c * (NB + 1) + m]);
    A[row * P + k0 + c] = s;
  }
}

// Trailing update A[r][c] -= sum_m X[r][m] conj(X[c][m]) on lower 64x64 tiles.
template <typename C>
__global__ void __launch_bounds__(256) k_herk(C* __restrict__ A, int64_t P, int64_t k0, int kw) {
  extern __shared__ unsigned char hsm[];
  C* Xr = reinterpret_cast<C*>(hsm);           // [NB (m)][NB+1 (row)]
  C* Xc = Xr + NB * (NB + 1);                  // [NB (m)][NB+1 (col)]
  const int64_t k1 = k0 + kw;
  // lower-triangular tile enumeration
  const int64_t t = blockIdx.x;
  int64_t tm = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
  while (tm * (tm + 1) / 2 > t) --tm;
  const int64_t tn = t - tm * (tm + 1) / 2;
  const int64_t r0 = k1 + tm * NB, c0 = k1 + tn * NB;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += 256) {
    const int rr = e / NB, m = e % NB;
    const int64_t row = r0 + rr, col = c0 + rr;
    Xr[m * (NB + 1) + rr] = (row < P && m < kw) ? A[row * P + k0 + m] : mk<C>(0.0, 0.0);
    Xc[m * (NB + 1) + rr] = (col < P && m < kw) ? A[col * P + k0 + m] : mk<C>(0.0, 0.0);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  C acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = mk<C>(0.0, 0.0);
  for (int m = 0; m < kw; ++m) {
    C xr[4], xc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xr[a] = Xr[m * (NB + 1) + ty + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) xc[b] = Xc[m * (NB + 1) + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) cfmac(acc[a][b], xr[a], xc[b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t row = r0 + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t col = c0 + tx + 16 * b;
      if (row < P && col < P && col <= row) {
        C v = A[row * P + col];
        v.x -= acc[a][b].x;
        v.y -= acc[a][b].y;
        A[row * P + col] = v;
      }
    }
  }
}

// Forward step kb of L y = b: y_kb = Linv_kb b_kb (every block recomputes it; block 0
// stores it), then b[r] -= sum_m L[r][k0+m] y_kb[m] for the rows below.
template <typename C>
__global__ void __launch_bounds__(256) k_fwd_step(const C* __restrict__ A,
                                                  const C* __restrict__ Dinv, int64_t P,
                                                  int64_t k0, int kw, C* __restrict__ b,
                                                  C* __restrict__ y) {
  __shared__ C yk[NB];
  const int tid = threadIdx.x;
  if (tid < kw) {
    C s = mk<C>(0.0, 0.0);
    for (int m = 0; m <= tid; ++m) cfma(s, Dinv[tid * NB + m], b[k0 + m]);
    yk[tid] = s;
    if (blockIdx.x == 0) y[k0 + tid] = s;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t first = k0 + kw;
  for (int64_t row = first + (int64_t)blockIdx.x * 8 + warp; row < P; row += (int64_t)gridDim.x * 8) {
    C s = mk<C>(0.0, 0.0);
    for (int m = lane; m < kw; m += 32) cfma(s, A[row * P + k0 + m], yk[m]);
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) {
      C v = b[row];
      v.x -= s.x;
      v.y -= s.y;
      b[row] = v;
    }
  }
}

// Backward step kb of L^H x = y: x_kb = Linv_kb^H c_kb, then c[r] -= sum_m conj(L[k0+m][r]) x_kb[m]
// for the rows above.
template <typename C>
__global__ void __launch_bounds__(256) k_bwd_step(const C* __restrict__ A,
                                                  const C* __restrict__ Dinv, int64_t P,
                                                  int64_t k0, int kw, C* __restrict__ c,
                                                  C* __restrict__ x) {
  __shared__ C xk[NB];
  const int tid = threadIdx.x;
  if (tid < kw) {
    C s = mk<C>(0.0, 0.0);
    for (int m = tid; m < kw; ++m) cfmac(s, c[k0 + m], Dinv[m * NB + tid]);  // conj(Linv[m][tid]) c[m]
    xk[tid] = s;
    if (blockIdx.x == 0) x[k0 + tid] = s;
  }
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + tid; r < k0; r += (int64_t)gridDim.x * blockDim.x) {
    C s = mk<C>(0.0, 0.0);
    for (int m = 0; m < kw; ++m) cfmac(s, xk[m], A[(k0 + m) * P + r]);
    C v = c[r];
    v.x -= s.x;
    v.y -= s.y;
    c[r] = v;
  }
}

// r = F - S~ x in FP64 (block per row), also |r|^2 accumulated into *acc
__global__ void __launch_bounds__(256) k_resid(const double2* __restrict__ S,
                                               const double2* __restrict__ x,
                                               const double2* __restrict__ F, int64_t P,
                                               double nu, int mode, double2* __restrict__ r,
                                               double* acc) {
  __shared__ double red[2][8];
  const int64_t row = blockIdx.x;
  double sr = 0.0, si = 0.0;
  for (int64_t c = threadIdx.x; c < P; c += blockDim.x) {
    const double2 a = S[row * P + c], v = x[c];
    sr = fma(a.x, v.x, sr);
    sr = fma(-a.y, v.y, sr);
    si = fma(a.x, v.y, si);
    si = fma(a.y, v.x, si);
  }
  sr = warp_sum_d(sr);
  si = warp_sum_d(si);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[0][w] = sr; red[1][w] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0, ti = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { tr += red[0][k]; ti += red[1][k]; }
    const double2 d = S[row * P + row], v = x[row];
    const double extra = (mode == 0) ? nu * d.x : nu;   // shift acts on the diagonal only
    tr += extra * v.x;
    ti += extra * v.y;
    const double2 f = F[row];
    const double2 res = make_double2(f.x - tr, f.y - ti);
    r[row] = res;
    atomicAdd(acc, res.x * res.x + res.y * res.y);
  }
}

__global__ void k_norm2(const double2* __restrict__ v, int64_t P, double* acc) {
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = v[k];
    s += a.x * a.x + a.y * a.y;
  }
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

__global__ void k_to_f32(const double2* __restrict__ a, float2* __restrict__ b, int64_t P) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x)
    b[k] = make_float2((float)a[k].x, (float)a[k].y);
}

__global__ void k_add_f32(double2* __restrict__ x, const float2* __restrict__ c, int64_t P) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    x[k].x += (double)c[k].x;
    x[k].y += (double)c[k].y;
  }
}

__global__ void k_update(double2* __restrict__ p, const double2* __restrict__ x, int64_t P, double dt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    p[k].x -= dt * x[k].x;
    p[k].y -= dt * x[k].y;
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
template <typename C>
static cudaError_t set_smem_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  const int s2 = 2 * NB * (NB + 1) * (int)sizeof(C);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_potrf_diag<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_trsm_inv<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_herk<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2)) != cudaSuccess) return e;
  done = true;
  return cudaSuccess;
}

static int grid_for(int64_t n, int threads, int cap = 8192) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

#define VMC_TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return _e; } while (0)

template <typename C>
static cudaError_t factor(C* A, C* Dinv, int64_t P, unsigned* status, cudaStream_t st,
                          int64_t* launches) {
  VMC_TRY(set_smem_attrs<C>());
  const size_t s2 = 2 * NB * (NB + 1) * sizeof(C);
  const int64_t nblk = (P + NB - 1) / NB;
  for (int64_t kb = 0; kb < nblk; ++kb) {
    const int64_t k0 = kb * NB;
    const int kw = (int)std::min<int64_t>(NB, P - k0);
    k_potrf_diag<C><<<1, POTRF_THREADS, s2, st>>>(A, P, k0, kw, Dinv + kb * NB * NB, status);
    ++*launches;
    const int64_t rest = P - k0 - kw;
    if (rest > 0) {
      k_trsm_inv<C><<<(unsigned)((rest + NB - 1) / NB), 256, s2, st>>>(A, P, k0, kw, Dinv + kb * NB * NB);
      const int64_t nt = (rest + NB - 1) / NB;
      k_herk<C><<<(unsigned)(nt * (nt + 1) / 2), 256, s2, st>>>(A, P, k0, kw);
      *launches += 2;
    }
    VMC_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

// b is overwritten (workspace); the solution lands in x
template <typename C>
static cudaError_t chol_solve(const C* A, const C* Dinv, int64_t P, C* b, C* y, C* x,
                              cudaStream_t st, int64_t* launches) {
  const int64_t nblk = (P + NB - 1) / NB;
  for (int64_t kb = 0; kb < nblk; ++kb) {
    const int64_t k0 = kb * NB;
    const int kw = (int)std::min<int64_t>(NB, P - k0);
    const int64_t rest = P - k0 - kw;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((rest + 7) / 8, 1184));
    k_fwd_step<C><<<g, 256, 0, st>>>(A, Dinv + kb * NB * NB, P, k0, kw, b, y);
    ++*launches;
  }
  for (int64_t kb = nblk - 1; kb >= 0; --kb) {
    const int64_t k0 = kb * NB;
    const int kw = (int)std::min<int64_t>(NB, P - k0);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((k0 + 255) / 256, 1184));
    k_bwd_step<C><<<g, 256, 0, st>>>(A, Dinv + kb * NB * NB, P, k0, kw, y, x);
    ++*launches;
  }
  return cudaGetLastError();
}

cudaError_t residual_fp64(const double2* S, const double2* F, const double2* x, double nu,
                          int mode, SolveWork& w, cudaStream_t st, double* relres) {
  const int64_t P = w.P;
  VMC_TRY(cudaMemsetAsync(w.scal, 0, 2 * sizeof(double), st));
  k_resid<<<(unsigned)P, 256, 0, st>>>(S, x, F, P, nu, mode, w.r, w.scal);
  k_norm2<<<grid_for(P, 256, 1024), 256, 0, st>>>(F, P, w.scal + 1);
  VMC_TRY(cudaGetLastError());
  double h[2];
  VMC_TRY(cudaMemcpyAsync(h, w.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  VMC_TRY(cudaStreamSynchronize(st));
  *relres = (h[1] > 0) ? sqrt(h[0] / h[1]) : 0.0;
  return cudaSuccess;
}

cudaError_t solve_cholesky_fp64(const double2* S, const double2* F, double2* x, double nu,
                                int mode, SolveWork& w, unsigned* status, cudaStream_t st,
                                int64_t* launches) {
  const int64_t P = w.P;
  k_copy_shift<double2><<<grid_for(P * P, 256), 256, 0, st>>>(S, w.A64, P, nu, mode);
  ++*launches;
  VMC_TRY(factor<double2>(w.A64, w.D64, P, status, st, launches));
  VMC_TRY(cudaMemcpyAsync(w.c, F, P * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  return chol_solve<double2>(w.A64, w.D64, P, w.c, w.r, x, st, launches);
}

cudaError_t solve_cholesky_mixed(const double2* S, const double2* F, double2* x, double nu,
                                 int mode, double tol, int maxit, SolveWork& w,
                                 unsigned* status, cudaStream_t st, int64_t* launches,
                                 int* iters, double* relres) {
  const int64_t P = w.P;
  k_copy_shift<float2><<<grid_for(P * P, 256), 256, 0, st>>>(S, w.A32, P, nu, mode);
  ++*launches;
  VMC_TRY(factor<float2>(w.A32, w.D32, P, status, st, launches));
  VMC_TRY(cudaMemsetAsync(x, 0, P * sizeof(double2), st));
  VMC_TRY(cudaMemcpyAsync(w.r, F, P * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  double rel = 1.0;
  int it = 0;
  for (; it < std::max(1, maxit); ++it) {
    k_to_f32<<<grid_for(P, 256, 1024), 256, 0, st>>>(w.r, w.r32, P);
    VMC_TRY(chol_solve<float2>(w.A32, w.D32, P, w.r32, w.y32, w.c32, st, launches));
    k_add_f32<<<grid_for(P, 256, 1024), 256, 0, st>>>(x, w.c32, P);
    *launches += 2;
    VMC_TRY(residual_fp64(S, F, x, nu, mode, w, st, &rel));
    *launches += 2;
    if (!(rel == rel)) break;      // NaN
    if (rel <= tol) { ++it; break; }
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;      // the caller compares it with tol
  return cudaSuccess;
}

cudaError_t launch_update(double2* params, const double2* x, int64_t P, double dt,
                          cudaStream_t st) {
  k_update<<<grid_for(P, 256, 4096), 256, 0, st>>>(params, x, P, dt);
  return cudaGetLastError();
}

}  // namespace vmc
