// cg.cu -- matrix-free conjugate gradient for S~ x = F (section "Diagonal shift": the
// shift combines with iterative solvers such as CG), used when S is too large to store.
//
// With O_q = [s_q | t_q | t_q (x) s_q] and Obar = O - <O>, for a vector v = [v_a | v_b | V]
// (V the W-block as an M x N matrix):
//   (Obar v)_q = s_q . v_a + t_q . (v_b + V s_q) - <O> . v            (one V S^T product)
//   (Obar^H u)_k / Ns = (1/Ns) sum_q conj(Obar_qk) u_q                 (the F reduction
//                                                                      with E_loc := u)
//   diag(S)_k = Var(O_k): 1 - <s_i>^2, <|t_j|^2> - |<t_j>|^2, <|t_j|^2> - |<t_j s_i>|^2
// so S~ v = (1/Ns) Obar^H (Obar v) + D v with D = nu diag(S) (multiplicative shift) or nu.
// The iteration is CG preconditioned with the diagonal of S~ (Jacobi): the diagonal spans
// orders of magnitude between the a-block (Var s ~ 1) and the b/W blocks (|t|^2 << 1).
// x, r, z, p, q and every dot product are FP64.
#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

// ---------------------------------------------------------------------------------------
// u_q = sum_j t_qj (v_b,j + sum_i V_ji s_qi) + sum_i s_qi v_a,i - c, as partial sums over
// 64-hidden tiles: part[mt][q].  Block: 64 samples x 64 hidden, K = N in steps of 32.
// ---------------------------------------------------------------------------------------
constexpr int VS_Q = 64, VS_J = 64, VS_K = 32;

__global__ void __launch_bounds__(256) k_vs_partial(const float2* __restrict__ V,  // [M][N]
                                                    const float2* __restrict__ vb, // [M]
                                                    const int8_t* __restrict__ spins,
                                                    const float2* __restrict__ T,  // [n][M]
                                                    int64_t n, int N, int M,
                                                    float2* __restrict__ part) {   // [mt][n]
  __shared__ float2 Vs[VS_J][VS_K + 1];
  __shared__ float Ss[VS_Q][VS_K + 1];
  __shared__ float2 red[VS_J / 4][VS_Q + 1];
  const int tid = threadIdx.x;
  const int64_t q0 = (int64_t)blockIdx.x * VS_Q;
  const int j0 = blockIdx.y * VS_J;
  const int tq = tid & 15, tj = tid >> 4;        // thread owns q = tq + 16 a, j = tj + 16 b
  float2 z[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) z[a][b] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < N; k0 += VS_K) {
    for (int e = tid; e < VS_J * VS_K; e += 256) {
      const int jj = e / VS_K, kk = e % VS_K;
      const int j = j0 + jj, i = k0 + kk;
      Vs[jj][kk] = (j < M && i < N) ? V[(int64_t)j * N + i] : make_float2(0.f, 0.f);
    }
    for (int e = tid; e < VS_Q * VS_K; e += 256) {
      const int qq = e / VS_K, kk = e % VS_K;
      const int64_t q = q0 + qq;
      const int i = k0 + kk;
      Ss[qq][kk] = (q < n && i < N) ? (float)spins[q * N + i] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < VS_K; ++kk) {
      float sv[4];
      float2 vv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) sv[a] = Ss[tq + 16 * a][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) vv[b] = Vs[tj + 16 * b][kk];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          z[a][b].x = fmaf(sv[a], vv[b].x, z[a][b].x);
          z[a][b].y = fmaf(sv[a], vv[b].y, z[a][b].y);
        }
    }
    __syncthreads();
  }
  // sum over this thread's hidden units of t_qj (vb_j + z_jq), then over the 16 row groups
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t q = q0 + tq + 16 * a;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tj + 16 * b;
      if (q < n && j < M) {
        const float2 w = make_float2(z[a][b].x + vb[j].x, z[a][b].y + vb[j].y);
        const float2 t = T[q * M + j];
        const float2 p = cmul(t, w);
        acc.x += p.x;
        acc.y += p.y;
      }
    }
    red[tj][tq + 16 * a] = acc;
  }
  __syncthreads();
  if (tid < VS_Q) {
    float2 acc = make_float2(0.f, 0.f);
    for (int g = 0; g < VS_J / 4; ++g) {
      acc.x += red[g][tid].x;
      acc.y += red[g][tid].y;
    }
    const int64_t q = q0 + tid;
    if (q < n) part[(int64_t)blockIdx.y * n + q] = acc;
  }
}

// u_q = sum_mt part[mt][q] + s_q . v_a - c   (c = <O> . v, from dev scalar)
__global__ void k_vs_finish(const float2* __restrict__ part, int mtiles, const int8_t* __restrict__ spins,
                            const float2* __restrict__ va, const double* __restrict__ c,
                            int64_t n, int N, float2* __restrict__ u) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    float ur = 0.f, ui = 0.f;
    for (int m = 0; m < mtiles; ++m) {
      const float2 p = part[(int64_t)m * n + q];
      ur += p.x;
      ui += p.y;
    }
    for (int i = 0; i < N; ++i) {
      const float s = (float)spins[q * N + i];
      ur = fmaf(s, va[i].x, ur);
      ui = fmaf(s, va[i].y, ui);
    }
    u[q] = make_float2(ur - (float)c[0], ui - (float)c[1]);
  }
}

// FP64 helpers -------------------------------------------------------------------------
constexpr int RED_BLOCKS = 256;

// partial[b] = sum over the block's slice of conj(a_k) b_k (complex), two-stage reduction
__global__ void __launch_bounds__(256) k_cdot_partial(const double2* __restrict__ a,
                                                      const double2* __restrict__ b, int64_t P,
                                                      double2* __restrict__ partial) {
  __shared__ double red[2][8];
  double sr = 0, si = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = a[k], y = b[k];
    sr += x.x * y.x + x.y * y.y;
    si += x.x * y.y - x.y * y.x;
  }
  sr = warp_sum_d(sr);
  si = warp_sum_d(si);
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sr; red[1][threadIdx.x >> 5] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0, ti = 0;
    for (int w = 0; w < 8; ++w) { tr += red[0][w]; ti += red[1][w]; }
    partial[blockIdx.x] = make_double2(tr, ti);
  }
}

// one warp: lane l adds partials l, l + 32, ...; then a fixed-order warp reduction
__global__ void k_cdot_final(const double2* __restrict__ partial, int nb, double2* __restrict__ out) {
  double tr = 0, ti = 0;
  for (int k = threadIdx.x; k < nb; k += 32) { tr += partial[k].x; ti += partial[k].y; }
  tr = warp_sum_d(tr);
  ti = warp_sum_d(ti);
  if (threadIdx.x == 0) *out = make_double2(tr, ti);
}

// mean of a complex FP32 vector in FP64: block partials, then one warp (fixed order)
__global__ void __launch_bounds__(256) k_mean_partial(const float2* __restrict__ u, int64_t n,
                                                      double2* __restrict__ partial) {
  __shared__ double red[2][8];
  double sr = 0, si = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = u[k];
    sr += v.x;
    si += v.y;
  }
  sr = warp_sum_d(sr);
  si = warp_sum_d(si);
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sr; red[1][threadIdx.x >> 5] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0, ti = 0;
    for (int w = 0; w < 8; ++w) { tr += red[0][w]; ti += red[1][w]; }
    partial[blockIdx.x] = make_double2(tr, ti);
  }
}

__global__ void k_mean_final(const double2* __restrict__ partial, int nb, int64_t n,
                             double* __restrict__ out) {
  double tr = 0, ti = 0;
  for (int k = threadIdx.x; k < nb; k += 32) { tr += partial[k].x; ti += partial[k].y; }
  tr = warp_sum_d(tr);
  ti = warp_sum_d(ti);
  if (threadIdx.x == 0) {
    out[0] = tr / (double)n;
    out[1] = ti / (double)n;
  }
}

// u_q = sum over the tiles' partials - c (the a block came through the product)
__global__ void k_vs_finish_tc(const float2* __restrict__ part, int mtiles,
                               const double* __restrict__ c, int64_t n, float2* __restrict__ u) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    float ur = 0.f, ui = 0.f;
    for (int m = 0; m < mtiles; ++m) {
      const float2 p = part[(int64_t)m * n + q];
      ur += p.x;
      ui += p.y;
    }
    u[q] = make_float2(ur - (float)c[0], ui - (float)c[1]);
  }
}

// diag(S) in closed form (s_i^2 = 1); t2[j] = <|t_j|^2>.  D = shift part, Minv = 1/diag(S~).
__global__ void k_diag_s(const double2* __restrict__ meanO, const double* __restrict__ t2, int N,
                         int M, double nu, int mode, double* __restrict__ D,
                         double* __restrict__ Minv) {
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 m = meanO[k];
    double v;
    if (k < N) v = 1.0 - (m.x * m.x + m.y * m.y);
    else if (k < N + M) v = t2[k - N] - (m.x * m.x + m.y * m.y);
    else v = t2[(k - N - M) / N] - (m.x * m.x + m.y * m.y);
    D[k] = (mode == 0) ? nu * v : nu;
    const double dd = v + D[k];
    Minv[k] = (dd > 0.0) ? 1.0 / dd : 1.0;
  }
}

// z = Minv r
__global__ void k_prec(const double* __restrict__ Minv, const double2* __restrict__ r, int64_t P,
                       double2* __restrict__ z) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x)
    z[k] = make_double2(Minv[k] * r[k].x, Minv[k] * r[k].y);
}

// t2[j] = (1/n) sum_q |t_qj|^2 in FP64
__global__ void k_t2(const float2* __restrict__ T, int64_t n, int M, double* __restrict__ t2) {
  const int j = blockIdx.x;
  __shared__ double red[8];
  double s = 0;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
    const float2 t = T[q * M + j];
    s += (double)t.x * t.x + (double)t.y * t.y;
  }
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    t2[j] = tot / (double)n;
  }
}

// split p into FP32 pieces for the product: va [N], vb [M], V [M][N] (row-major as in p)
__global__ void k_split_v(const double2* __restrict__ p, int N, int M, float2* __restrict__ va,
                          float2* __restrict__ vb, float2* __restrict__ V) {
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const float2 f = make_float2((float)p[k].x, (float)p[k].y);
    if (k < N) va[k] = f;
    else if (k < N + M) vb[k - N] = f;
    else V[k - N - M] = f;
  }
}

// q = y + D p
__global__ void k_add_diag(const double2* __restrict__ y, const double* __restrict__ D,
                           const double2* __restrict__ p, int64_t P, double2* __restrict__ q) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x)
    q[k] = make_double2(y[k].x + D[k] * p[k].x, y[k].y + D[k] * p[k].y);
}

// x += alpha p; r -= alpha q
__global__ void k_cg_xr(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
                        const double2* __restrict__ q, int64_t P, const double* __restrict__ alpha) {
  const double al = *alpha;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    x[k].x += al * p[k].x;
    x[k].y += al * p[k].y;
    r[k].x -= al * q[k].x;
    r[k].y -= al * q[k].y;
  }
}

// p = r + beta p
__global__ void k_cg_p(double2* __restrict__ p, const double2* __restrict__ r, int64_t P,
                       const double* __restrict__ beta) {
  const double be = *beta;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x)
    p[k] = make_double2(r[k].x + be * p[k].x, r[k].y + be * p[k].y);
}

// scalars: sc[0] = r.z, sc[1] = p.q (re), sc[2] = alpha, sc[3] = beta, sc[4] = new r.z,
// sc[5] = |r|^2
__global__ void k_cg_alpha(double* sc, const double2* pq) {
  sc[1] = pq->x;
  sc[2] = (pq->x != 0.0) ? sc[0] / pq->x : 0.0;
}
__global__ void k_cg_beta(double* sc, const double2* rz_new, const double2* rr) {
  sc[4] = rz_new->x;
  sc[3] = (sc[0] != 0.0) ? sc[4] / sc[0] : 0.0;
  sc[0] = sc[4];
  sc[5] = rr->x;
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
#define VMC_TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return _e; } while (0)

static int g1d(int64_t n, int cap = 4096) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, cap));
}

int64_t cg_partial_floats2(int64_t n, int M) { return ((M + VS_J - 1) / VS_J) * n; }

static cudaError_t cdot(const double2* a, const double2* b, int64_t P, CgWork& w, double2* out,
                        cudaStream_t st) {
  k_cdot_partial<<<RED_BLOCKS, 256, 0, st>>>(a, b, P, w.dpart);
  k_cdot_final<<<1, 32, 0, st>>>(w.dpart, RED_BLOCKS, out);
  return cudaGetLastError();
}

// q = S~ p
// ---------------------------------------------------------------------------------------
// Tensor-core operator.  Per step: Sb = spins as BF16 [q][i] (A of the Obar v product) and
// Bs = [spins^T ; ones] [i][q] (B of the Obar^H u product); per CG iteration: the direction's
// W block as hi/lo real-row planes, and A2 = [conj(t_qj)(u_q - <u>) rows 2j / 2j+1 ; (u_q -
// <u>) rows 2M / 2M+1] as hi/lo planes [row][q].  Zero padding everywhere the products
// read (K padding must be finite: 0 x garbage could be NaN).
// ---------------------------------------------------------------------------------------
static inline int64_t pad_to(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

__global__ void k_build_sb(const int8_t* __restrict__ spins, int64_t n, int N, int64_t rows,
                           int64_t K, __nv_bfloat16* __restrict__ Sb) {
  const int64_t total = rows * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / K;
    const int i = (int)(e - q * K);
    Sb[e] = __float2bfloat16_rn((q < n && i < N) ? (float)spins[q * N + i] : 0.f);
  }
}

// Bs[i][q] (32 x 32 tiles through shared memory)
__global__ void k_build_bs(const int8_t* __restrict__ spins, int64_t n, int N, int64_t rows,
                           int64_t K, __nv_bfloat16* __restrict__ Bs) {
  __shared__ float tile[32][33];
  const int64_t q0 = (int64_t)blockIdx.x * 32;
  const int i0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t q = q0 + r;
    const int i = i0 + tx;
    float v = 0.f;
    if (q < n) v = (i < N) ? (float)spins[q * N + i] : (i == N ? 1.f : 0.f);
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r;
    const int64_t q = q0 + tx;
    if (i < rows && q < K) Bs[(int64_t)i * K + q] = __float2bfloat16_rn(tile[tx][r]);
  }
}

// rows 2j / 2j+1: Re / Im of V_j (j < M); rows 2M / 2M+1: Re / Im of v_a
__global__ void k_build_vplanes(const float2* __restrict__ V, const float2* __restrict__ va,
                                int N, int M, int64_t rows, int64_t K,
                                __nv_bfloat16* __restrict__ Vhi, __nv_bfloat16* __restrict__ Vlo) {
  const int64_t total = rows * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / K;
    const int i = (int)(e - r * K);
    const int j = (int)(r >> 1);
    float v = 0.f;
    if (j <= M && i < N) {
      const float2 z = (j < M) ? V[(int64_t)j * N + i] : va[i];
      v = (r & 1) ? z.y : z.x;
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Vhi[e] = h;
    Vlo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// A2 rows [2j, 2j+1] = conj(t_qj) u'_q, rows [2M, 2M+1] = u'_q, u' = u - mean(u)
__global__ void k_build_a2(const float2* __restrict__ T, const float2* __restrict__ u,
                           const double* __restrict__ ustats, int64_t n, int M, int64_t rows,
                           int64_t K, __nv_bfloat16* __restrict__ Ahi,
                           __nv_bfloat16* __restrict__ Alo) {
  __shared__ float2 tile[32][33];
  const int64_t q0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;                 // complex row index (j or M for u')
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const float mr = (float)ustats[0], mi = (float)ustats[1];
  for (int r = ty; r < 32; r += 8) {
    const int64_t q = q0 + r;
    const int j = j0 + tx;
    float2 w = make_float2(0.f, 0.f);
    if (q < n) {
      const float2 uq = u[q];
      const float ur = uq.x - mr, ui = uq.y - mi;
      if (j < M) {
        const float2 t = T[q * M + j];
        w = make_float2(t.x * ur + t.y * ui, t.x * ui - t.y * ur);   // conj(t) u'
      } else if (j == M) {
        w = make_float2(ur, ui);
      }
    }
    tile[r][tx] = w;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r;
    const int64_t q = q0 + tx;
    if (2 * (int64_t)j + 1 < rows && q < K) {
      const float2 w = tile[tx][r];
      const __nv_bfloat16 hr = __float2bfloat16_rn(w.x), hi = __float2bfloat16_rn(w.y);
      Ahi[(2 * (int64_t)j) * K + q] = hr;
      Ahi[(2 * (int64_t)j + 1) * K + q] = hi;
      Alo[(2 * (int64_t)j) * K + q] = __float2bfloat16_rn(w.x - __bfloat162float(hr));
      Alo[(2 * (int64_t)j + 1) * K + q] = __float2bfloat16_rn(w.y - __bfloat162float(hi));
    }
  }
}

// y_k = (1/n) sum_q conj(Obar_qk) u_q from the K-chunk partials G[kc][row][col] (FP64 sum):
// a_i: rows 2M/2M+1, col i; b_j: rows 2j/2j+1, col N; W_ji: rows 2j/2j+1, col i
// four threads per entry (chunks c = q, q + 4, ...), then a fixed-order shuffle sum
__global__ void __launch_bounds__(256) k_reduce_y(const float* __restrict__ part, int nkc,
                                                  int64_t a_rows, int64_t b_rows, int N, int M,
                                                  int64_t n, double2* __restrict__ y) {
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  const double inv = 1.0 / (double)n;
  const int64_t k = (int64_t)blockIdx.x * 64 + (threadIdx.x >> 2);
  const int q = threadIdx.x & 3;
  double re = 0.0, im = 0.0;
  if (k < P) {
    int64_t row, col;
    if (k < N) { row = 2 * (int64_t)M; col = k; }
    else if (k < N + M) { row = 2 * (k - N); col = N; }
    else { const int64_t r = k - N - M; row = 2 * (r / N); col = r % N; }
    for (int c = q; c < nkc; c += 4) {
      const float* g = part + (int64_t)c * a_rows * b_rows;
      re += (double)g[row * b_rows + col];
      im += (double)g[(row + 1) * b_rows + col];
    }
  }
  re += __shfl_xor_sync(0xffffffffu, re, 1);
  im += __shfl_xor_sync(0xffffffffu, im, 1);
  re += __shfl_xor_sync(0xffffffffu, re, 2);
  im += __shfl_xor_sync(0xffffffffu, im, 2);
  if (k < P && q == 0) y[k] = make_double2(re * inv, im * inv);
}

static cudaError_t apply_s_tc(const CgProblem& pb, CgWork& w, const double2* p, double2* q,
                              cudaStream_t st, int64_t* launches) {
  const int N = pb.N, M = pb.M;
  const int64_t n = pb.n, P = (int64_t)N + M + (int64_t)N * M;
  const int64_t kN = pad_to(N, 64), s_rows = pad_to(n, 128), v_rows = pad_to(2 * (int64_t)M + 2, 128);
  const int64_t ldK = pad_to(n, 64), a_rows = pad_to(2 * (int64_t)M + 2, 128),
                b_rows = pad_to((int64_t)N + 1, 128);
  const int nkc = (int)((ldK / 64 + CG_KB_PER_CHUNK - 1) / CG_KB_PER_CHUNK);
  if (v_rows * kN > w.cap_v || a_rows * ldK > w.cap_a || nkc * a_rows * b_rows > w.cap_part2)
    return cudaErrorInvalidValue;
  k_split_v<<<g1d(P), 256, 0, st>>>(p, N, M, w.va, w.vb, w.V);
  k_build_vplanes<<<g1d(v_rows * kN), 256, 0, st>>>(w.V, w.va, N, M, v_rows, kN, w.Vhi, w.Vlo);
  VMC_TRY(cdot(pb.meanO_conj_free, p, P, w, w.c2, st));   // c = sum_k <O_k> p_k (no conj)
  VMC_TRY(launch_cg_ov_tc(w.Sb, s_rows, kN, w.Vhi, w.Vlo, v_rows, pb.T, w.vb, M, n, w.upart,
                          pb.status, st));
  const int mtiles = (int)(v_rows / 128);
  k_vs_finish_tc<<<g1d(n), 256, 0, st>>>(w.upart, mtiles, reinterpret_cast<const double*>(w.c2),
                                         n, w.u);
  {
    const int nb = (int)std::min<int64_t>(RED_BLOCKS, (n + 1023) / 1024);
    k_mean_partial<<<nb, 256, 0, st>>>(w.u, n, w.dpart);
    k_mean_final<<<1, 32, 0, st>>>(w.dpart, nb, n, w.ustats);
  }
  dim3 ga((unsigned)(ldK / 32), (unsigned)((a_rows / 2 + 31) / 32));
  k_build_a2<<<ga, 256, 0, st>>>(pb.T, w.u, w.ustats, n, M, a_rows, ldK, w.Ahi, w.Alo);
  VMC_TRY(launch_cg_ohu_tc(w.Ahi, w.Alo, a_rows, w.Bs, b_rows, ldK, CG_KB_PER_CHUNK, w.part2,
                           pb.status, st));
  k_reduce_y<<<(unsigned)((P + 63) / 64), 256, 0, st>>>(w.part2, nkc, a_rows, b_rows, N, M, n, w.y);
  k_add_diag<<<g1d(P), 256, 0, st>>>(w.y, w.D, p, P, q);
  *launches += 12;
  return cudaGetLastError();
}

static cudaError_t apply_s(const CgProblem& pb, CgWork& w, const double2* p, double2* q,
                           cudaStream_t st, int64_t* launches) {
  if (pb.tc) return apply_s_tc(pb, w, p, q, st, launches);
  const int N = pb.N, M = pb.M;
  const int64_t n = pb.n, P = (int64_t)N + M + (int64_t)N * M;
  k_split_v<<<g1d(P), 256, 0, st>>>(p, N, M, w.va, w.vb, w.V);
  VMC_TRY(cdot(pb.meanO_conj_free, p, P, w, w.c2, st));   // c = sum_k <O_k> p_k (no conj)
  const int mtiles = (M + VS_J - 1) / VS_J;
  dim3 grid((unsigned)((n + VS_Q - 1) / VS_Q), (unsigned)mtiles);
  k_vs_partial<<<grid, 256, 0, st>>>(w.V, w.vb, pb.spins, pb.T, n, N, M, w.upart);
  k_vs_finish<<<g1d(n), 256, 0, st>>>(w.upart, mtiles, pb.spins, w.va,
                                      reinterpret_cast<const double*>(w.c2), n, N, w.u);
  VMC_TRY(launch_estats(w.u, n, w.ustats, nullptr, st));
  VMC_TRY(launch_moments(pb.spins, pb.T, w.u, w.ustats, n, N, M, w.mpart, nullptr, w.y, st));
  k_add_diag<<<g1d(P), 256, 0, st>>>(w.y, w.D, p, P, q);
  *launches += 11;
  return cudaGetLastError();
}

__global__ void k_conj_copy(const double2* __restrict__ a, int64_t P, double2* __restrict__ b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x)
    b[k] = make_double2(a[k].x, -a[k].y);
}

cudaError_t cg_prepare(const CgProblem& pb, CgWork& w, double nu, int mode, cudaStream_t st,
                       int64_t* launches) {
  const int64_t P = (int64_t)pb.N + pb.M + (int64_t)pb.N * pb.M;
  k_t2<<<pb.M, 256, 0, st>>>(pb.T, pb.n, pb.M, w.t2);
  k_diag_s<<<g1d(P), 256, 0, st>>>(pb.meanO, w.t2, pb.N, pb.M, nu, mode, w.D, w.Minv);
  // <O> with conjugation undone so that cdot(conj(a), p) gives sum <O_k> p_k
  k_conj_copy<<<g1d(P), 256, 0, st>>>(pb.meanO, P, w.meanO_c);
  *launches += 3;
  if (pb.tc) {
    const int64_t kN = pad_to(pb.N, 64), s_rows = pad_to(pb.n, 128), ldK = pad_to(pb.n, 64);
    const int64_t b_rows = pad_to((int64_t)pb.N + 1, 128);
    if (s_rows * kN > w.cap_sb || b_rows * ldK > w.cap_bs) return cudaErrorInvalidValue;
    k_build_sb<<<g1d(s_rows * kN), 256, 0, st>>>(pb.spins, pb.n, pb.N, s_rows, kN, w.Sb);
    dim3 gb((unsigned)(ldK / 32), (unsigned)(b_rows / 32));
    k_build_bs<<<gb, 256, 0, st>>>(pb.spins, pb.n, pb.N, b_rows, ldK, w.Bs);
    *launches += 2;
  }
  return cudaGetLastError();
}

cudaError_t cg_solve(const CgProblem& pb_in, const double2* F, double2* x, double tol, int maxit,
                     CgWork& w, cudaStream_t st, int64_t* launches, int* iters, double* relres) {
  CgProblem pb = pb_in;
  pb.meanO_conj_free = w.meanO_c;
  const int64_t P = (int64_t)pb.N + pb.M + (int64_t)pb.N * pb.M;
  VMC_TRY(cudaMemsetAsync(x, 0, P * sizeof(double2), st));
  VMC_TRY(cudaMemsetAsync(w.sc, 0, 8 * sizeof(double), st));
  VMC_TRY(cudaMemcpyAsync(w.r, F, P * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  k_prec<<<g1d(P), 256, 0, st>>>(w.Minv, w.r, P, w.z);
  VMC_TRY(cudaMemcpyAsync(w.p, w.z, P * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  VMC_TRY(cdot(w.r, w.z, P, w, w.c2 + 1, st));
  VMC_TRY(cdot(w.r, w.r, P, w, w.c2 + 4, st));
  k_cg_beta<<<1, 1, 0, st>>>(w.sc, w.c2 + 1, w.c2 + 4);     // sc[0] = r.z, sc[5] = |F|^2
  *launches += 6;
  double h[8];
  VMC_TRY(cudaMemcpyAsync(h, w.sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  VMC_TRY(cudaStreamSynchronize(st));
  const double f2 = h[5];
  double rr = f2;
  int it = 0;
  while (it < maxit && rr > tol * tol * f2) {
    VMC_TRY(apply_s(pb, w, w.p, w.q, st, launches));
    VMC_TRY(cdot(w.p, w.q, P, w, w.c2 + 2, st));
    k_cg_alpha<<<1, 1, 0, st>>>(w.sc, w.c2 + 2);
    k_cg_xr<<<g1d(P), 256, 0, st>>>(x, w.r, w.p, w.q, P, w.sc + 2);
    k_prec<<<g1d(P), 256, 0, st>>>(w.Minv, w.r, P, w.z);
    VMC_TRY(cdot(w.r, w.z, P, w, w.c2 + 3, st));
    VMC_TRY(cdot(w.r, w.r, P, w, w.c2 + 5, st));
    k_cg_beta<<<1, 1, 0, st>>>(w.sc, w.c2 + 3, w.c2 + 5);
    k_cg_p<<<g1d(P), 256, 0, st>>>(w.p, w.z, P, w.sc + 3);
    *launches += 12;
    VMC_TRY(cudaMemcpyAsync(h, w.sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    VMC_TRY(cudaStreamSynchronize(st));
    rr = h[5];
    ++it;
    if (!(rr == rr)) break;
  }
  if (iters) *iters = it;
  if (relres) *relres = (f2 > 0) ? sqrt(rr / f2) : 0.0;
  return cudaGetLastError();
}

}  // namespace vmc
