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
// Tensor-core operator (products in cg_tc.cu).  Per step: Sb = spins as BF16 [q][i] (A of
// the Obar v product) and Bs = spins^T [i][q] (B of the Obar^H u product); per CG
// iteration: the direction's W block and v_a as hi/lo real-row planes.  Zero padding
// everywhere the products read (K padding must be finite: 0 x garbage could be NaN).
// ---------------------------------------------------------------------------------------
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
    tile[r][tx] = (q < n && i < N) ? (float)spins[q * N + i] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r;
    const int64_t q = q0 + tx;
    if (i < rows && q < K) Bs[(int64_t)i * K + q] = __float2bfloat16_rn(tile[tx][r]);
  }
}

// Re / Im of V_j (j < M) and of v_a (the pseudo-unit j = M), rows in the order the
// product's epilogue reads them: within each block of 32 rows (16 units), row
// 8k + 2 cq + c holds component c of unit 4 cq + k, so that the 16x256b TMEM load gives a
// thread four consecutive units.
__global__ void k_build_vplanes(const float2* __restrict__ V, const float2* __restrict__ va,
                                int N, int M, int64_t rows, int64_t K,
                                __nv_bfloat16* __restrict__ Vhi, __nv_bfloat16* __restrict__ Vlo) {
  const int64_t total = rows * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / K;
    const int i = (int)(e - r * K);
    const int rho = (int)(r & 31);
    const int j = (int)(r >> 5) * 16 + 4 * ((rho & 7) >> 1) + (rho >> 3);
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

// q_k = y_k + D_k p_k with y_k = (1/n) sum_q conj(Obar_qk) w_q from the K-chunk partials
// (FP64 sum over chunks): a_i: out rows 2M / 2M+1, column i; b_j: ybpart[.][j]; W_ji: out
// rows 2j / 2j+1, column i.  Four threads per entry (chunks c = l, l + 4, ...), then a
// fixed-order shuffle sum.
__global__ void __launch_bounds__(256) k_cg_reduce_tc(const float* __restrict__ out,
                                                      const float2* __restrict__ ybpart,
                                                      int kchunks, int64_t a_rows, int ncols,
                                                      int N, int M, int64_t n,
                                                      const double* __restrict__ D,
                                                      const double2* __restrict__ p,
                                                      double2* __restrict__ q) {
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  const double inv = 1.0 / (double)n;
  const int64_t k = (int64_t)blockIdx.x * 64 + (threadIdx.x >> 2);
  const int l = threadIdx.x & 3;
  double re = 0.0, im = 0.0;
  if (k < P) {
    if (k >= N && k < N + M) {
      for (int c = l; c < kchunks; c += 4) {
        const float2 v = ybpart[(int64_t)c * M + (k - N)];
        re += (double)v.x;
        im += (double)v.y;
      }
    } else {
      int64_t row, col;
      if (k < N) { row = 2 * (int64_t)M; col = k; }
      else { const int64_t r = k - N - M; row = 2 * (r / N); col = r % N; }
      for (int c = l; c < kchunks; c += 4) {
        const float* g = out + (int64_t)c * a_rows * ncols;
        re += (double)g[row * ncols + col];
        im += (double)g[(row + 1) * ncols + col];
      }
    }
  }
  re += __shfl_xor_sync(0xffffffffu, re, 1);
  im += __shfl_xor_sync(0xffffffffu, im, 1);
  re += __shfl_xor_sync(0xffffffffu, re, 2);
  im += __shfl_xor_sync(0xffffffffu, im, 2);
  if (k < P && l == 0) {
    const double2 pk = p[k];
    q[k] = make_double2(re * inv + D[k] * pk.x, im * inv + D[k] * pk.y);
  }
}

static cudaError_t apply_s_tc(const CgProblem& pb, CgWork& w, const double2* p, double2* q,
                              cudaStream_t st, int64_t* launches) {
  const int N = pb.N, M = pb.M;
  const int64_t n = pb.n, P = (int64_t)N + M + (int64_t)N * M;
  const CgTcShape sh = cg_tc_shape(N, M, n);
  if (!sh.ok || sh.v_rows * sh.kN > w.cap_v ||
      (int64_t)sh.kchunks * sh.mtiles * 128 * sh.nbt * 128 > w.cap_part2 ||
      (int64_t)sh.kchunks * M > w.cap_yb)
    return cudaErrorInvalidValue;
  k_split_v<<<g1d(P), 256, 0, st>>>(p, N, M, w.va, w.vb, w.V);
  k_build_vplanes<<<g1d(sh.v_rows * sh.kN), 256, 0, st>>>(w.V, w.va, N, M, sh.v_rows, sh.kN,
                                                          w.Vhi, w.Vlo);
  VMC_TRY(cdot(pb.meanO_conj_free, p, P, w, w.c2, st));   // c = sum_k <O_k> p_k (no conj)
  int nup = 0;
  VMC_TRY(launch_cg_ov_tc(w.Sb, w.Vhi, w.Vlo, sh, pb.T, w.vb, reinterpret_cast<const double*>(w.c2),
                          M, n, w.u, w.ovpart, &nup, pb.status, st));
  if (nup > w.cap_ov) return cudaErrorInvalidValue;
  VMC_TRY(launch_cg_ohu_tc(w.Bs, sh, pb.T, w.u, w.ovpart, nup, M, n, w.part2, w.ybpart,
                           pb.status, st));
  k_cg_reduce_tc<<<(unsigned)((P + 63) / 64), 256, 0, st>>>(w.part2, w.ybpart, sh.kchunks,
                                                            (int64_t)sh.mtiles * 128, sh.nbt * 128,
                                                            N, M, n, w.D, p, q);
  *launches += 7;
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
    const CgTcShape sh = cg_tc_shape(pb.N, pb.M, pb.n);
    if (!sh.ok || sh.s_rows * sh.kN > w.cap_sb || sh.b_rows * sh.ldK > w.cap_bs)
      return cudaErrorInvalidValue;
    k_build_sb<<<g1d(sh.s_rows * sh.kN), 256, 0, st>>>(pb.spins, pb.n, pb.N, sh.s_rows, sh.kN,
                                                       w.Sb);
    dim3 gb((unsigned)(sh.ldK / 32), (unsigned)(sh.b_rows / 32));
    k_build_bs<<<gb, 256, 0, st>>>(pb.spins, pb.n, pb.N, sh.b_rows, sh.ldK, w.Bs);
    *launches += 2;
  }
  return cudaGetLastError();
}

cudaError_t cg_apply(const CgProblem& pb_in, CgWork& w, const double2* v, double2* y,
                     cudaStream_t st, int64_t* launches) {
  CgProblem pb = pb_in;
  pb.meanO_conj_free = w.meanO_c;
  return apply_s(pb, w, v, y, st, launches);
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
