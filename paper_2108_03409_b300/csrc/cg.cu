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

// t2[j] = (1/n) sum_q |t_qj|^2 in FP64: block b sums rows b, b + T2_BLOCKS, ... (threads
// along j, coalesced), then one thread per j adds the T2_BLOCKS partials in order
constexpr int T2_BLOCKS = 256;
__global__ void __launch_bounds__(256) k_t2_partial(const float2* __restrict__ T, int64_t n,
                                                    int M, double* __restrict__ part) {
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double s = 0.0;
    for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
      const float2 t = T[q * M + j];
      s += (double)t.x * t.x + (double)t.y * t.y;
    }
    part[(int64_t)blockIdx.x * M + j] = s;
  }
}

__global__ void k_t2_final(const double* __restrict__ part, int nb, int64_t n, int M,
                           double* __restrict__ t2) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * M + j];
    t2[j] = s / (double)n;
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
#define VMC_TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return _e; } while (0)

static int g1d(int64_t n, int cap = 4096) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, cap));
}

int64_t cg_partial_floats2(int64_t n, int M) { return ((M + VS_J - 1) / VS_J) * n; }

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
// thread four consecutive units.  Read from the FP64 direction p (rounded to FP32, then
// split); vb = v_b in FP32 for the epilogue.
__global__ void k_build_vplanes(const double2* __restrict__ p, int N, int M, int64_t rows,
                                int64_t K, __nv_bfloat16* __restrict__ Vhi,
                                __nv_bfloat16* __restrict__ Vlo, float2* __restrict__ vb,
                                const int* __restrict__ done) {
  if (*done) return;
  const int64_t total = rows * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / K;
    const int i = (int)(e - r * K);
    const int rho = (int)(r & 31);
    const int j = (int)(r >> 5) * 16 + 4 * ((rho & 7) >> 1) + (rho >> 3);
    float v = 0.f;
    if (j <= M && i < N) {
      const double2 z = (j < M) ? p[N + M + (int64_t)j * N + i] : p[i];
      v = (float)((rho & 1) ? z.y : z.x);
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Vhi[e] = h;
    Vlo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    if (e < M) vb[e] = make_float2((float)p[N + e].x, (float)p[N + e].y);
  }
}

// ---------------------------------------------------------------------------------------
// CG vector kernels.  Every reduction is a fixed-order FP64 sum: each of CG_VB blocks
// writes one partial, and whoever needs the total sums the CG_VB partials in a fixed order
// (lane l takes l, l + 32, ..., then the warp tree).  Partial buffers (doubles):
//   PQ   Re p^H q                     written by the operator's last kernel
//   RZ   Re r^H z, two buffers by iteration parity (the update writes one, reads the other)
//   RR   |r|^2, two buffers by iteration parity
//   CR/CI  sum_k <O_k> p_k (no conjugation): the centring constant of Obar p
// Scalars sc: [0] |F|^2, [1] |r|^2 of the latest check, [2..3] c = <O> . p.
// Flags: [0] done (converged or non-finite), [1] iterations performed.
// ---------------------------------------------------------------------------------------
constexpr int CG_VB = 256;             // blocks of the vector kernels
constexpr int CG_RB = 1024;            // blocks of the chunk reduction (its p.q partials)
constexpr int OFF_PQ = 0, OFF_RZ = 1024, OFF_RR = 1536, OFF_CR = 2048, OFF_CI = 2304;
static_assert(OFF_CI + CG_VB <= CG_VPART_DOUBLES, "CG partial buffer");

// sum of NP partials, lane l taking l, l + 32, ... (all loads issued before the adds)
template <int NP>
__device__ __forceinline__ double sum_partials(const double* part, int lane) {
  double v[NP / 32];
#pragma unroll
  for (int k = 0; k < NP / 32; ++k) v[k] = part[lane + 32 * k];
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NP / 32; ++k) s += v[k];
  return warp_sum_d(s);
}

// block sum of one value per thread (up to 256 threads) into part[blockIdx.x]
__device__ __forceinline__ void block_partial(double v, double* part, double* red) {
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
  __syncthreads();
}

// x = 0, r = F, z = Minv r, p = z; partials of r.z (parity slot 1), |r|^2 (slot 1), <O>.p
__global__ void __launch_bounds__(256) k_cg_init(const double2* __restrict__ F,
                                                 const double* __restrict__ Minv,
                                                 const double2* __restrict__ meanO, int64_t P,
                                                 double2* __restrict__ x, double2* __restrict__ r,
                                                 double2* __restrict__ z, double2* __restrict__ p,
                                                 double* __restrict__ vpart) {
  __shared__ double red[8];
  double rz = 0.0, rr = 0.0, cr = 0.0, ci = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double2 f = F[k];
    const double2 zk = make_double2(Minv[k] * f.x, Minv[k] * f.y);
    x[k] = make_double2(0.0, 0.0);
    r[k] = f;
    z[k] = zk;
    p[k] = zk;
    rz += f.x * zk.x + f.y * zk.y;
    rr += f.x * f.x + f.y * f.y;
    const double2 m = meanO[k];
    cr += m.x * zk.x - m.y * zk.y;
    ci += m.x * zk.y + m.y * zk.x;
  }
  block_partial(rz, vpart + OFF_RZ + CG_VB, red);
  block_partial(rr, vpart + OFF_RR + CG_VB, red);
  block_partial(cr, vpart + OFF_CR, red);
  block_partial(ci, vpart + OFF_CI, red);
}

// start of iteration `it` (one warp): |r|^2 and c from the partials of the previous
// update / direction kernels; sets done once |r|^2 <= tol2 |F|^2 (or non-finite), else
// counts the iteration (if `count`).  Nothing changes once done is set, so sc[1] keeps the
// residual at which the iteration stopped.
__global__ void k_cg_check(const double* __restrict__ vpart, int it, double tol2, double* sc,
                           int* flag, int first, int count) {
  if (flag[0]) return;
  const int lane = threadIdx.x;
  const int prev = (it & 1) ^ 1;
  const double rr = sum_partials<CG_VB>(vpart + OFF_RR + prev * CG_VB, lane);
  const double cr = sum_partials<CG_VB>(vpart + OFF_CR, lane);
  const double ci = sum_partials<CG_VB>(vpart + OFF_CI, lane);
  if (lane == 0) {
    if (first) sc[0] = rr;
    sc[1] = rr;
    sc[2] = cr;
    sc[3] = ci;
    const double f2 = first ? rr : sc[0];
    if (!(rr > tol2 * f2) || !(rr == rr)) flag[0] = 1;
    else if (count) flag[1] += 1;
  }
}

// alpha = r.z / p.q; x += alpha p; r -= alpha q; z = Minv r; partials of r.z and |r|^2
__global__ void __launch_bounds__(256) k_cg_update(double2* __restrict__ x, double2* __restrict__ r,
                                                   double2* __restrict__ z,
                                                   const double2* __restrict__ p,
                                                   const double2* __restrict__ q,
                                                   const double* __restrict__ Minv, int64_t P,
                                                   double* __restrict__ vpart, int it,
                                                   const int* __restrict__ done) {
  if (*done) return;
  __shared__ double red[8];
  __shared__ double alpha_s;
  const int par = it & 1;
  if (threadIdx.x < 32) {
    const double rz = sum_partials<CG_VB>(vpart + OFF_RZ + (par ^ 1) * CG_VB, threadIdx.x);
    const double pq = sum_partials<CG_RB>(vpart + OFF_PQ, threadIdx.x);
    if (threadIdx.x == 0) alpha_s = (pq != 0.0) ? rz / pq : 0.0;
  }
  __syncthreads();
  const double al = alpha_s;
  double rz = 0.0, rr = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double2 pk = p[k], qk = q[k];
    double2 xk = x[k], rk = r[k];
    xk.x += al * pk.x;
    xk.y += al * pk.y;
    rk.x -= al * qk.x;
    rk.y -= al * qk.y;
    x[k] = xk;
    r[k] = rk;
    const double2 zk = make_double2(Minv[k] * rk.x, Minv[k] * rk.y);
    z[k] = zk;
    rz += rk.x * zk.x + rk.y * zk.y;
    rr += rk.x * rk.x + rk.y * rk.y;
  }
  block_partial(rz, vpart + OFF_RZ + par * CG_VB, red);
  block_partial(rr, vpart + OFF_RR + par * CG_VB, red);
}

// beta = r.z (new) / r.z (old); p = z + beta p; partials of <O>.p for the next operator
__global__ void __launch_bounds__(256) k_cg_dir(double2* __restrict__ p,
                                                const double2* __restrict__ z,
                                                const double2* __restrict__ meanO, int64_t P,
                                                double* __restrict__ vpart, int it,
                                                const int* __restrict__ done) {
  if (*done) return;
  __shared__ double red[8];
  __shared__ double beta_s;
  const int par = it & 1;
  if (threadIdx.x < 32) {
    const double rz_new = sum_partials<CG_VB>(vpart + OFF_RZ + par * CG_VB, threadIdx.x);
    const double rz_old = sum_partials<CG_VB>(vpart + OFF_RZ + (par ^ 1) * CG_VB, threadIdx.x);
    if (threadIdx.x == 0) beta_s = (rz_old != 0.0) ? rz_new / rz_old : 0.0;
  }
  __syncthreads();
  const double be = beta_s;
  double cr = 0.0, ci = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double2 zk = z[k], pk = p[k];
    const double2 pn = make_double2(zk.x + be * pk.x, zk.y + be * pk.y);
    p[k] = pn;
    const double2 m = meanO[k];
    cr += m.x * pn.x - m.y * pn.y;
    ci += m.x * pn.y + m.y * pn.x;
  }
  block_partial(cr, vpart + OFF_CR, red);
  block_partial(ci, vpart + OFF_CI, red);
}

// partials of <O>.v for one application of the operator to v
__global__ void __launch_bounds__(256) k_cg_cpart(const double2* __restrict__ v,
                                                  const double2* __restrict__ meanO, int64_t P,
                                                  double* __restrict__ vpart) {
  __shared__ double red[8];
  double cr = 0.0, ci = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double2 m = meanO[k], pk = v[k];
    cr += m.x * pk.x - m.y * pk.y;
    ci += m.x * pk.y + m.y * pk.x;
  }
  block_partial(cr, vpart + OFF_CR, red);
  block_partial(ci, vpart + OFF_CI, red);
}

// SIMT operator: FP32 copies of the direction
__global__ void k_split_v(const double2* __restrict__ p, int N, int M, float2* __restrict__ va,
                          float2* __restrict__ vb, float2* __restrict__ V,
                          const int* __restrict__ done) {
  if (*done) return;
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const float2 f = make_float2((float)p[k].x, (float)p[k].y);
    if (k < N) va[k] = f;
    else if (k < N + M) vb[k - N] = f;
    else V[k - N - M] = f;
  }
}

// q = y + D p, with partials of Re p^H q
__global__ void __launch_bounds__(256) k_add_diag(const double2* __restrict__ y,
                                                  const double* __restrict__ D,
                                                  const double2* __restrict__ p, int64_t P,
                                                  double2* __restrict__ q,
                                                  double* __restrict__ vpart,
                                                  const int* __restrict__ done) {
  if (*done) return;
  __shared__ double red[8];
  double pq = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 pk = p[k];
    const double2 qk = make_double2(y[k].x + D[k] * pk.x, y[k].y + D[k] * pk.y);
    q[k] = qk;
    pq += pk.x * qk.x + pk.y * qk.y;
  }
  block_partial(pq, vpart + OFF_PQ, red);
}

constexpr int RED_U = 16;   // chunk partials of one entry loaded together

// q_k = y_k + D_k p_k with y_k = (1/n) sum_q conj(Obar_qk) w_q from the K-chunk partials
// (compensated sum over chunks in order): a_i: out rows 2M / 2M+1, column i; b_j: ybpart[.][j];
// W_ji: out rows 2j / 2j+1, column i.  Partials of Re p^H q.  Without D: q = y (conjugated
// if conj_out), no partials.
__global__ void __launch_bounds__(128) k_cg_reduce_tc(const float* __restrict__ out,
                                                      const float2* __restrict__ ybpart,
                                                      int kchunks, int64_t a_rows, int ncols,
                                                      int N, int M, int64_t n,
                                                      const double* __restrict__ D,
                                                      const double2* __restrict__ p,
                                                      double2* __restrict__ q,
                                                      double* __restrict__ vpart,
                                                      const int* __restrict__ done,
                                                      int conj_out) {
  if (*done) return;
  __shared__ double red[8];
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
  const double inv = 1.0 / (double)n;
  double pq = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    // the chunk partials of entry k, RED_U chunks at a time: all their loads are issued
    // before the (in-order, compensated) sums, so that a thread keeps 2 RED_U loads in flight
    CSum sr, si;
    const float* g;
    int64_t cs, off_im;
    if (k >= N && k < N + M) {
      g = reinterpret_cast<const float*>(ybpart + (k - N));
      cs = 2 * (int64_t)M;
      off_im = 1;
    } else {
      int64_t row, col;
      if (k < N) { row = 2 * (int64_t)M; col = k; }
      else { const int rr = (int)(k - N - M); row = 2 * (int64_t)(rr / N); col = rr % N; }
      g = out + row * ncols + col;
      cs = a_rows * ncols;
      off_im = ncols;
    }
    for (int c0 = 0; c0 < kchunks; c0 += RED_U) {
      float vr[RED_U], vi[RED_U];
#pragma unroll
      for (int u = 0; u < RED_U; ++u) {
        const int64_t o = (int64_t)min(c0 + u, kchunks - 1) * cs;
        vr[u] = __ldg(g + o);
        vi[u] = __ldg(g + o + off_im);
      }
#pragma unroll
      for (int u = 0; u < RED_U; ++u)
        if (c0 + u < kchunks) {
          sr.add(vr[u]);
          si.add(vi[u]);
        }
    }
    const double re = sr.value(), im = si.value();
    if (D) {
      const double2 pk = p[k];
      const double2 qk = make_double2(re * inv + D[k] * pk.x, im * inv + D[k] * pk.y);
      q[k] = qk;
      pq += pk.x * qk.x + pk.y * qk.y;
    } else {
      q[k] = make_double2(re * inv, conj_out ? -im * inv : im * inv);
    }
  }
  if (D) block_partial(pq, vpart + OFF_PQ, red);
}

static cudaError_t apply_s_tc(const CgProblem& pb, CgWork& w, const double2* p, double2* q,
                              cudaStream_t st, int64_t* launches) {
  const int N = pb.N, M = pb.M;
  const int64_t n = pb.n;
  const CgTcShape sh = cg_tc_shape(N, M, n);
  if (!sh.ok || sh.v_rows * sh.kN > w.cap_v ||
      (int64_t)sh.kchunks * sh.mtiles * 128 * sh.nbt * 128 > w.cap_part2 ||
      (int64_t)sh.kchunks * M > w.cap_yb)
    return cudaErrorInvalidValue;
  k_build_vplanes<<<g1d(sh.v_rows * sh.kN), 256, 0, st>>>(p, N, M, sh.v_rows, sh.kN, w.Vhi,
                                                          w.Vlo, w.vb, w.flag);
  int nup = 0;
  VMC_TRY(launch_cg_ov_tc(w.Sb, w.Vhi, w.Vlo, sh, pb.T, w.vb, w.sc + 2, M, n, w.u, w.ovpart,
                          &nup, w.flag, pb.status, st));
  if (nup > w.cap_ov) return cudaErrorInvalidValue;
  VMC_TRY(launch_cg_ohu_tc(w.Bs, sh, pb.T, w.u, w.ovpart, nup, nullptr, M, n, w.part2, w.ybpart,
                           w.flag, pb.status, st));
  k_cg_reduce_tc<<<CG_RB, 128, 0, st>>>(w.part2, w.ybpart, sh.kchunks, (int64_t)sh.mtiles * 128,
                                        sh.nbt * 128, N, M, n, w.D, p, q, w.vpart, w.flag, 0);
  *launches += 4;
  return cudaGetLastError();
}

// q = S~ p with the centring constant c = <O>.p already in w.sc[2..3]
static cudaError_t apply_s(const CgProblem& pb, CgWork& w, const double2* p, double2* q,
                           cudaStream_t st, int64_t* launches) {
  if (pb.tc) return apply_s_tc(pb, w, p, q, st, launches);
  const int N = pb.N, M = pb.M;
  const int64_t n = pb.n, P = (int64_t)N + M + (int64_t)N * M;
  k_split_v<<<g1d(P), 256, 0, st>>>(p, N, M, w.va, w.vb, w.V, w.flag);
  const int mtiles = (M + VS_J - 1) / VS_J;
  dim3 grid((unsigned)((n + VS_Q - 1) / VS_Q), (unsigned)mtiles);
  k_vs_partial<<<grid, 256, 0, st>>>(w.V, w.vb, pb.spins, pb.T, n, N, M, w.upart);
  k_vs_finish<<<g1d(n), 256, 0, st>>>(w.upart, mtiles, pb.spins, w.va, w.sc + 2, n, N, w.u);
  VMC_TRY(launch_estats(w.u, n, w.ustats, nullptr, st));
  VMC_TRY(launch_moments(pb.spins, pb.T, w.u, w.ustats, n, N, M, w.mpart, nullptr, w.y, st));
  k_add_diag<<<CG_RB, 256, 0, st>>>(w.y, w.D, p, P, q, w.vpart, w.flag);
  *launches += 8;
  return cudaGetLastError();
}

__global__ void k_fill_ones(float2* __restrict__ a, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    a[k] = make_float2(1.f, 0.f);
}

cudaError_t fill_ones(float2* a, int64_t n) {
  k_fill_ones<<<g1d(n), 256>>>(a, n);
  return cudaGetLastError();
}

// the spin operands of the tensor-core products (Sb [q][i] and Bs = Sb^T), once per sample set
static cudaError_t build_spin_operands(const CgProblem& pb, CgWork& w, cudaStream_t st,
                                       int64_t* launches) {
  const CgTcShape sh = cg_tc_shape(pb.N, pb.M, pb.n);
  if (!sh.ok || sh.s_rows * sh.kN > w.cap_sb || sh.b_rows * sh.ldK > w.cap_bs)
    return cudaErrorInvalidValue;
  k_build_sb<<<g1d(sh.s_rows * sh.kN), 256, 0, st>>>(pb.spins, pb.n, pb.N, sh.s_rows, sh.kN, w.Sb);
  dim3 gb((unsigned)(sh.ldK / 32), (unsigned)(sh.b_rows / 32));
  k_build_bs<<<gb, 256, 0, st>>>(pb.spins, pb.n, pb.N, sh.b_rows, sh.ldK, w.Bs);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t cg_moments_tc(const CgProblem& pb, const float2* E, const double* estats,
                          double2* meanO, double2* F, CgWork& w, cudaStream_t st,
                          int64_t* launches) {
  VMC_TRY(build_spin_operands(pb, w, st, launches));
  const int N = pb.N, M = pb.M;
  const int64_t n = pb.n, P = (int64_t)N + M + (int64_t)N * M;
  const CgTcShape sh = cg_tc_shape(N, M, n);
  if ((int64_t)sh.kchunks * sh.mtiles * 128 * sh.nbt * 128 > w.cap_part2 ||
      (int64_t)sh.kchunks * M > w.cap_yb)
    return cudaErrorInvalidValue;
  const int* zero = w.flag + 4;
  // F_k = (1/n) sum_q conj(O_qk) (E_q - <E>)
  VMC_TRY(launch_cg_ohu_tc(w.Bs, sh, pb.T, E, nullptr, 0, estats, M, n, w.part2, w.ybpart, zero,
                           pb.status, st));
  k_cg_reduce_tc<<<CG_RB, 128, 0, st>>>(w.part2, w.ybpart, sh.kchunks, (int64_t)sh.mtiles * 128,
                                        sh.nbt * 128, N, M, n, nullptr, nullptr, F, nullptr, zero, 0);
  // <O_k> = conj((1/n) sum_q conj(O_qk) 1)
  VMC_TRY(launch_cg_ohu_tc(w.Bs, sh, pb.T, w.ones, nullptr, 0, w.zero2, M, n, w.part2, w.ybpart,
                           zero, pb.status, st));
  k_cg_reduce_tc<<<CG_RB, 128, 0, st>>>(w.part2, w.ybpart, sh.kchunks, (int64_t)sh.mtiles * 128,
                                        sh.nbt * 128, N, M, n, nullptr, nullptr, meanO, nullptr, zero,
                                        1);
  *launches += 4;
  (void)P;
  return cudaGetLastError();
}

cudaError_t cg_prepare(const CgProblem& pb, CgWork& w, double nu, int mode, cudaStream_t st,
                       int64_t* launches, bool operands_ready) {
  const int64_t P = (int64_t)pb.N + pb.M + (int64_t)pb.N * pb.M;
  static_assert(T2_BLOCKS == CG_T2_BLOCKS, "t2 partial buffer");
  k_t2_partial<<<T2_BLOCKS, 256, 0, st>>>(pb.T, pb.n, pb.M, w.t2part);
  k_t2_final<<<(pb.M + 255) / 256, 256, 0, st>>>(w.t2part, T2_BLOCKS, pb.n, pb.M, w.t2);
  k_diag_s<<<g1d(P), 256, 0, st>>>(pb.meanO, w.t2, pb.N, pb.M, nu, mode, w.D, w.Minv);
  *launches += 3;
  // the spin operands, unless cg_moments_tc just built them for this sample set
  if (pb.tc && !operands_ready) VMC_TRY(build_spin_operands(pb, w, st, launches));
  return cudaGetLastError();
}

cudaError_t cg_apply(const CgProblem& pb, CgWork& w, const double2* v, double2* y,
                     cudaStream_t st, int64_t* launches) {
  const int64_t P = (int64_t)pb.N + pb.M + (int64_t)pb.N * pb.M;
  VMC_TRY(cudaMemsetAsync(w.flag, 0, 4 * sizeof(int), st));
  k_cg_cpart<<<CG_VB, 256, 0, st>>>(v, pb.meanO, P, w.vpart);
  // the check kernel publishes c (its |r|^2 and done outputs are not used here)
  k_cg_check<<<1, 32, 0, st>>>(w.vpart, 0, 0.0, w.sc, w.flag + 2, 1, 0);
  *launches += 2;
  return apply_s(pb, w, v, y, st, launches);
}

// Host loop: the iterations are enqueued without waiting; every CG_SYNC_EVERY iterations
// the host reads the done flag.  Iterations enqueued after convergence find done set and
// return at once, so the result equals that of a check after every iteration.
constexpr int CG_SYNC_EVERY = 4;

cudaError_t cg_solve(const CgProblem& pb, const double2* F, double2* x, double tol, int maxit,
                     CgWork& w, cudaStream_t st, int64_t* launches, int* iters, double* relres) {
  const int64_t P = (int64_t)pb.N + pb.M + (int64_t)pb.N * pb.M;
  const double tol2 = tol * tol;
  VMC_TRY(cudaMemsetAsync(w.flag, 0, 4 * sizeof(int), st));
  k_cg_init<<<CG_VB, 256, 0, st>>>(F, w.Minv, pb.meanO, P, x, w.r, w.z, w.p, w.vpart);
  *launches += 1;
  int h_flag[4] = {0, 0, 0, 0};
  for (int it = 0; it < maxit; ++it) {
    k_cg_check<<<1, 32, 0, st>>>(w.vpart, it, tol2, w.sc, w.flag, it == 0, 1);
    VMC_TRY(apply_s(pb, w, w.p, w.q, st, launches));
    k_cg_update<<<CG_VB, 256, 0, st>>>(x, w.r, w.z, w.p, w.q, w.Minv, P, w.vpart, it, w.flag);
    k_cg_dir<<<CG_VB, 256, 0, st>>>(w.p, w.z, pb.meanO, P, w.vpart, it, w.flag);
    *launches += 3;
    if ((it + 1) % CG_SYNC_EVERY == 0 && it + 1 < maxit) {
      VMC_TRY(cudaMemcpyAsync(h_flag, w.flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
      VMC_TRY(cudaStreamSynchronize(st));
      if (h_flag[0]) break;
    }
  }
  // the residual of the final state when maxit ended the loop (a no-op once done is set)
  k_cg_check<<<1, 32, 0, st>>>(w.vpart, maxit, tol2, w.sc, w.flag, maxit == 0, 0);
  *launches += 1;
  double h_sc[4];
  VMC_TRY(cudaMemcpyAsync(h_sc, w.sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  VMC_TRY(cudaMemcpyAsync(h_flag, w.flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  VMC_TRY(cudaStreamSynchronize(st));
  if (iters) *iters = h_flag[1];
  if (relres) *relres = (h_sc[0] > 0) ? sqrt(h_sc[1] / h_sc[0]) : 0.0;
  return cudaGetLastError();
}

}  // namespace vmc
