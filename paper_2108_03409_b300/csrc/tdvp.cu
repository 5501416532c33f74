// tdvp.cu -- the regularised TDVP right-hand side (arXiv:2108.03409, sections "Unitary
// dynamics" and "Regularization to invert the (quantum) Fisher matrix"):
//   weighted <E>, <O>, F and the Fisher matrix S (Eq. qfm, Eq. force_vector) in FP64,
//   the eigen-decomposition S = V diag(lambda) V^H (parallel cyclic Jacobi, FP64),
//   rho = V^H F, the SNR of every rho_k from the energy-weighted Gram Q, the damped
//   inverse eigenvalues lambda^+ (Eq. pinv_cutoff or its soft form, times the SNR damping),
//   and thetadot = -gamma V (lambda^+ rho);
// plus the vector kernels of the adaptive Heun integrator and the Fisher norm.
//
// Samples carry weights w (the Born weights p(s) for exact enumeration, or none: 1/n).
// Everything after the FP32 inputs (spins, t = tanh theta, E_loc) is FP64: the pseudo-
// inverse divides by eigenvalues down to eps_pinv * lambda_1, which FP32 sums of products
// would bury in rounding.
#include <cmath>

#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

namespace {

constexpr int kTile = 32;          // Gram tile (32 x 32 entries)
constexpr int kBatch = 32;         // samples staged per round in the Gram kernel

__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconjmul_d(double2 a, double2 b) {   // conj(a) * b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

// O_k(s) of the RBM (Eq. rbm_ex derivatives): s_i (k < N), t_j (k < N + M), t_j s_i.
__device__ __forceinline__ double2 o_entry(const int8_t* s, const float2* t, int N, int M,
                                           int64_t k) {
  if (k < N) return make_double2((double)s[k], 0.0);
  if (k < N + M) {
    const float2 v = t[k - N];
    return make_double2((double)v.x, (double)v.y);
  }
  const int64_t r = k - N - M;
  const int j = (int)(r / N), i = (int)(r % N);
  const float2 v = t[j];
  const double si = (double)s[i];
  return make_double2(si * (double)v.x, si * (double)v.y);
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {   // blockDim.x <= 1024, multiple of 32
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];   // same order in every thread
  return r;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = sh[0];
  for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, sh[k]);
  return r;
}

// ---------------------------------------------------------------------------------------
// exact enumeration (the ExactSampler of the "Sampler" section)
// ---------------------------------------------------------------------------------------
__global__ void k_enum_states(int8_t* spins, int N, int64_t n) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * N) return;
  const int64_t k = idx / N;
  const int i = (int)(idx % N);
  spins[idx] = ((k >> i) & 1) ? (int8_t)-1 : (int8_t)1;     // bit 0 <-> s = +1
}

// Born weights p(s) = exp(2 Re log psi(s) - 2 max) / sum (one block).
__global__ void k_born_weights(const float2* lp, int64_t n, double* w, unsigned* status) {
  __shared__ double sh[32];
  double m = -INFINITY;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) m = fmax(m, (double)lp[k].x);
  m = block_max(m, sh);
  double z = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double e = exp(2.0 * ((double)lp[k].x - m));
    w[k] = e;
    z += e;
  }
  z = block_sum(z, sh);
  if (!(z > 0.0) || !isfinite(z)) {
    if (threadIdx.x == 0) flag_error(status, DEV_ERR_NUMERIC);
    return;
  }
  const double inv = 1.0 / z;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) w[k] *= inv;
}

// w_out = w_in / sum(w_in) (one block); a non-positive or non-finite sum sets the status
// (sums, if given: sum w and sum w^2 of the input)
__global__ void k_normalize_weights(const double* w_in, int64_t n, double* w_out,
                                    unsigned* status, double* sums) {
  __shared__ double sh[32];
  double z = 0.0, z2 = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    z += w_in[k];
    z2 += w_in[k] * w_in[k];
  }
  z = block_sum(z, sh);
  z2 = block_sum(z2, sh);
  if (sums && threadIdx.x == 0) {
    sums[0] = z;
    sums[1] = z2;
  }
  if (!(z > 0.0) || !isfinite(z)) {
    if (threadIdx.x == 0) flag_error(status, DEV_ERR_NUMERIC);
    return;
  }
  const double inv = 1.0 / z;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) w_out[k] = w_in[k] * inv;
}

// ---------------------------------------------------------------------------------------
// weighted energy statistics: out[0..3] = <E>.re, <E>.im, <|E - <E>|^2>, stderr; one block.
// w == null: uniform weights 1/n (stderr = sqrt(var / n)); otherwise stderr = 0 (exact).
// ---------------------------------------------------------------------------------------
__global__ void k_tdvp_energy(const float2* E, const double* w, int64_t n, double* out,
                              unsigned* status) {
  __shared__ double sh[32];
  const double u = 1.0 / (double)n;
  double er = 0.0, ei = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double wk = w ? w[k] : u;
    er = fma(wk, (double)E[k].x, er);
    ei = fma(wk, (double)E[k].y, ei);
  }
  er = block_sum(er, sh);
  ei = block_sum(ei, sh);
  double v = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double wk = w ? w[k] : u;
    const double dr = (double)E[k].x - er, di = (double)E[k].y - ei;
    v = fma(wk, dr * dr + di * di, v);
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) {
    out[0] = er;
    out[1] = ei;
    out[2] = v;
    out[3] = w ? 0.0 : sqrt(v / (double)n);
    if (!isfinite(er) || !isfinite(ei) || !isfinite(v)) flag_error(status, DEV_ERR_NUMERIC);
  }
}

// weighted <O_k> and F_k = sum_s w conj(O_k(s)) (E(s) - <E>): thread per k, blockIdx.y a
// chunk of samples; partial[chunk][k] = {sum w O_k, sum w conj(O_k)(E - <E>)}.
__global__ void k_tdvp_moments(const int8_t* __restrict__ spins, const float2* __restrict__ T,
                               const float2* __restrict__ E, const double* __restrict__ w,
                               const float2* __restrict__ osc, const float* __restrict__ Od,
                               const double* __restrict__ estats, int64_t n, int N, int M,
                               int64_t P, int64_t chunk, double2* __restrict__ partial) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const int64_t q0 = (int64_t)blockIdx.y * chunk, q1 = min(n, q0 + chunk);
  const double u = 1.0 / (double)n;
  const double er = estats[0], ei = estats[1];
  double mr = 0, mi = 0, fr = 0, fi = 0;
  for (int64_t q = q0; q < q1; ++q) {
    const double wq = w ? w[q] : u;
    double2 o = Od ? make_double2((double)Od[q * P + k], 0.0)
                   : o_entry(spins + q * N, T + q * M, N, M, k);
    if (osc) o = cmul_d(o, make_double2((double)osc[q].x, (double)osc[q].y));
    const double dr = (double)E[q].x - er, di = (double)E[q].y - ei;
    mr = fma(wq, o.x, mr);
    mi = fma(wq, o.y, mi);
    // conj(o) (d) = (o.x d.x + o.y d.y) + i (o.x d.y - o.y d.x)
    fr = fma(wq, fma(o.x, dr, o.y * di), fr);
    fi = fma(wq, fma(o.x, di, -o.y * dr), fi);
  }
  partial[((int64_t)blockIdx.y * P + k) * 2 + 0] = make_double2(mr, mi);
  partial[((int64_t)blockIdx.y * P + k) * 2 + 1] = make_double2(fr, fi);
}

__global__ void k_tdvp_moments_reduce(const double2* __restrict__ partial, int chunks, int64_t P,
                                      double2* meanO, double2* F) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  double2 m = make_double2(0, 0), f = make_double2(0, 0);
  for (int c = 0; c < chunks; ++c) {
    const double2 a = partial[((int64_t)c * P + k) * 2 + 0];
    const double2 b = partial[((int64_t)c * P + k) * 2 + 1];
    m.x += a.x; m.y += a.y;
    f.x += b.x; f.y += b.y;
  }
  meanO[k] = m;
  F[k] = f;
}

// ---------------------------------------------------------------------------------------
// weighted Grams of the centred log-derivatives, lower 32 x 32 tiles:
//   S_kl = sum_s w conj(Obar_k) Obar_l,   Q_kl = sum_s w |E - <E>|^2 conj(Obar_k) Obar_l.
// blockIdx.x = lower tile, blockIdx.y = sample chunk; 256 threads, thread (ty, tx) owns
// row k = tile row + tx and columns l = tile col + 4 ty .. 4 ty + 3.  The Obar values of a
// batch of 32 samples are staged in shared memory (FP64).
// partial[chunk][tile][1024][2] (S, Q).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void tri_tile(int64_t t, int* bm, int* bn) {
  int m = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)m * (m + 1) / 2 > t) --m;
  while ((int64_t)(m + 1) * (m + 2) / 2 <= t) ++m;
  *bm = m;
  *bn = (int)(t - (int64_t)m * (m + 1) / 2);
}

__global__ void __launch_bounds__(256) k_tdvp_gram(
    const int8_t* __restrict__ spins, const float2* __restrict__ T, const float2* __restrict__ E,
    const double* __restrict__ w, const float2* __restrict__ osc, const float* __restrict__ Od,
    const double* __restrict__ estats, const double2* __restrict__ meanO, int64_t n, int N,
    int M, int64_t P, int64_t chunk, int64_t ntiles, double2* __restrict__ partial) {
  __shared__ double2 Ok[kBatch][kTile];
  __shared__ double2 Ol[kBatch][kTile];
  __shared__ double ws[kBatch], wq[kBatch];
  int bm, bn;
  tri_tile(blockIdx.x, &bm, &bn);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t k0 = (int64_t)bm * kTile, l0 = (int64_t)bn * kTile;
  const int64_t q0 = (int64_t)blockIdx.y * chunk, q1 = min(n, q0 + chunk);
  const double u = 1.0 / (double)n;
  const double er = estats[0], ei = estats[1];
  double2 s_acc[4], q_acc[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) { s_acc[c] = make_double2(0, 0); q_acc[c] = make_double2(0, 0); }
  for (int64_t qb = q0; qb < q1; qb += kBatch) {
    const int nb = (q1 - qb) < kBatch ? (int)(q1 - qb) : kBatch;
    __syncthreads();
    // stage: 2 * 32 * 32 values by 256 threads
    for (int e = threadIdx.x; e < 2 * kBatch * kTile; e += 256) {
      const int side = e / (kBatch * kTile);
      const int r = e % (kBatch * kTile);
      const int qs = r / kTile, c = r % kTile;
      const int64_t kk = (side ? l0 : k0) + c;
      double2 v = make_double2(0, 0);
      if (qs < nb && kk < P) {
        const int64_t q = qb + qs;
        double2 o = Od ? make_double2((double)Od[q * P + kk], 0.0)
                       : o_entry(spins + q * N, T + q * M, N, M, kk);
        if (osc) o = cmul_d(o, make_double2((double)osc[q].x, (double)osc[q].y));
        const double2 m = meanO[kk];
        v = make_double2(o.x - m.x, o.y - m.y);
      }
      if (side) Ol[qs][c] = v; else Ok[qs][c] = v;
    }
    if (threadIdx.x < kBatch) {
      const int qs = threadIdx.x;
      double a = 0.0, b = 0.0;
      if (qs < nb) {
        const int64_t q = qb + qs;
        a = w ? w[q] : u;
        const double dr = (double)E[q].x - er, di = (double)E[q].y - ei;
        b = a * (dr * dr + di * di);
      }
      ws[qs] = a;
      wq[qs] = b;
    }
    __syncthreads();
    for (int qs = 0; qs < nb; ++qs) {
      const double2 a = Ok[qs][tx];
      const double wa = ws[qs], wb = wq[qs];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double2 p = cconjmul_d(a, Ol[qs][4 * ty + c]);
        s_acc[c].x = fma(wa, p.x, s_acc[c].x);
        s_acc[c].y = fma(wa, p.y, s_acc[c].y);
        q_acc[c].x = fma(wb, p.x, q_acc[c].x);
        q_acc[c].y = fma(wb, p.y, q_acc[c].y);
      }
    }
  }
  double2* out = partial + (((int64_t)blockIdx.y * ntiles + blockIdx.x) * (kTile * kTile)) * 2;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int e = tx * kTile + 4 * ty + c;      // (row tx, column 4 ty + c)
    out[2 * e + 0] = s_acc[c];
    out[2 * e + 1] = q_acc[c];
  }
}

// sum of the chunk partials in a fixed order; writes the full Hermitian S and Q
__global__ void k_tdvp_gram_reduce(const double2* __restrict__ partial, int chunks, int64_t ntiles,
                                   int64_t P, double2* S, double2* Q) {
  const int64_t t = blockIdx.x;
  const int e = threadIdx.x;                  // 1024 threads: one tile entry each
  int bm, bn;
  tri_tile(t, &bm, &bn);
  const int64_t k = (int64_t)bm * kTile + e / kTile, l = (int64_t)bn * kTile + e % kTile;
  if (k >= P || l >= P || l > k) return;
  double2 s = make_double2(0, 0), q = make_double2(0, 0);
  for (int c = 0; c < chunks; ++c) {
    const double2* p = partial + (((int64_t)c * ntiles + t) * (kTile * kTile) + e) * 2;
    s.x += p[0].x; s.y += p[0].y;
    q.x += p[1].x; q.y += p[1].y;
  }
  if (k == l) { s.y = 0.0; q.y = 0.0; }
  S[k * P + l] = s;
  S[l * P + k] = make_double2(s.x, -s.y);
  Q[k * P + l] = q;
  Q[l * P + k] = make_double2(q.x, -q.y);
}

// ---------------------------------------------------------------------------------------
// Eigen-decomposition of a Hermitian matrix by the parallel cyclic Jacobi method (one
// cooperative launch).  n is padded to an even ne with an inert index.  Each round pairs
// every index once (round-robin: position 0 fixed, the others rotated), and
//   phase A: every pair (p, q) gets the unitary J = [[c, sigma], [-conj(sigma), c]] with
//            sigma = s e^{i arg A_pq}, t = s / c the smaller root of
//            t^2 + 2 tau t - 1 = 0, tau = (A_qq - A_pp) / (2 |A_pq|), which zeroes A_pq;
//   phase B: A <- J^H A J on every 2 x 2 block of the pair partition, V <- V J.
// A sweep is ne - 1 rounds; sweeps continue until the off-diagonal Frobenius norm is below
// tol times the matrix's.  Barriers are bounded; A, V and the rotations are read with
// L2-only loads (other blocks wrote them since the last barrier).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int rr_index(int pos, int r, int ne) {
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (ne - 1);
}

__device__ __forceinline__ double2 ld2(const double2* p) { return __ldcg(p); }

__device__ double grid_reduce_sum(double v, double* red, GridBarrier* bar, unsigned nb,
                                  unsigned* status, bool* ok) {
  __shared__ double sh[32];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) __stcg(red + blockIdx.x, v);
  if (!grid_sync(bar, nb, status)) { *ok = false; return 0.0; }
  double s = 0.0;
  for (unsigned b = 0; b < nb; ++b) s += __ldcg(red + b);   // same order in every block
  if (!grid_sync(bar, nb, status)) { *ok = false; return 0.0; }  // red reusable afterwards
  return s;
}

__global__ void __launch_bounds__(256) k_jacobi_eig(double2* A, double2* V, int n, int ne,
                                                    double* lam, double2* rot, GridBarrier* bar,
                                                    double* red, unsigned* status, int max_sweeps,
                                                    double tol, double* info) {
  const unsigned nb = gridDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int half = ne / 2;
  bool ok = true;
  double fro = 0.0;
  for (int64_t e = tid; e < (int64_t)n * n; e += nthr) {
    const int i = (int)(e / n), j = (int)(e % n);
    V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    const double2 a = A[e];
    fro += a.x * a.x + a.y * a.y;
  }
  fro = grid_reduce_sum(fro, red, bar, nb, status, &ok);
  if (!ok) return;
  int sweep = 0;
  double off = 0.0;
  for (; sweep <= max_sweeps; ++sweep) {
    off = 0.0;
    for (int64_t e = tid; e < (int64_t)n * n; e += nthr) {
      const int i = (int)(e / n), j = (int)(e % n);
      if (i == j) continue;
      const double2 a = ld2(A + e);
      off += a.x * a.x + a.y * a.y;
    }
    off = grid_reduce_sum(off, red, bar, nb, status, &ok);
    if (!ok) return;
    if (off <= tol * tol * fro || sweep == max_sweeps) break;
    for (int r = 0; r < ne - 1; ++r) {
      // phase A: rotations
      for (int64_t k = tid; k < half; k += nthr) {
        int p = rr_index((int)k, r, ne), q = rr_index(ne - 1 - (int)k, r, ne);
        if (p > q) { const int x = p; p = q; q = x; }
        double2 Rc = make_double2(1.0, 0.0), Rs = make_double2(0.0, 0.0);   // c; sigma
        if (q < n) {
          const double a = ld2(A + (int64_t)p * n + p).x, b = ld2(A + (int64_t)q * n + q).x;
          const double2 c = ld2(A + (int64_t)p * n + q);
          const double ac = hypot(c.x, c.y);
          if (ac > 1e-300 && ac > 1e-18 * sqrt(fabs(a) * fabs(b))) {
            const double tau = (b - a) / (2.0 * ac);
            const double t = (fabs(tau) > 1e150) ? 0.5 / tau
                             : copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
            Rc = make_double2(cs, 0.0);
            Rs = make_double2(sn * c.x / ac, sn * c.y / ac);
          }
        }
        __stcg(rot + 2 * k, Rc);
        __stcg(rot + 2 * k + 1, Rs);
      }
      if (!grid_sync(bar, nb, status)) return;
      // phase B: A <- J^H A J on 2 x 2 blocks, V <- V J
      const int64_t nblk = (int64_t)half * half;
      for (int64_t e = tid; e < nblk + (int64_t)n * half; e += nthr) {
        if (e < nblk) {
          const int ia = (int)(e / half), ib = (int)(e % half);
          int pa = rr_index(ia, r, ne), qa = rr_index(ne - 1 - ia, r, ne);
          if (pa > qa) { const int x = pa; pa = qa; qa = x; }
          int pb = rr_index(ib, r, ne), qb = rr_index(ne - 1 - ib, r, ne);
          if (pb > qb) { const int x = pb; pb = qb; qb = x; }
          const double ca = __ldcg(rot + 2 * ia).x, cb = __ldcg(rot + 2 * ib).x;
          const double2 sa = __ldcg(rot + 2 * ia + 1), sb = __ldcg(rot + 2 * ib + 1);
          const bool qa_ok = qa < n, qb_ok = qb < n;
          const double2 z = make_double2(0, 0);
          const double2 x00 = ld2(A + (int64_t)pa * n + pb);
          const double2 x01 = qb_ok ? ld2(A + (int64_t)pa * n + qb) : z;
          const double2 x10 = qa_ok ? ld2(A + (int64_t)qa * n + pb) : z;
          const double2 x11 = (qa_ok && qb_ok) ? ld2(A + (int64_t)qa * n + qb) : z;
          // Y = X Jb:  [x0, x1] Jb = [c x0 - conj(sig) x1, sig x0 + c x1]
          const double2 sbc = make_double2(sb.x, -sb.y);
          double2 y00 = cmul_d(sbc, x01), y10 = cmul_d(sbc, x11);
          y00 = make_double2(cb * x00.x - y00.x, cb * x00.y - y00.y);
          y10 = make_double2(cb * x10.x - y10.x, cb * x10.y - y10.y);
          double2 y01 = cmul_d(sb, x00), y11 = cmul_d(sb, x10);
          y01 = make_double2(y01.x + cb * x01.x, y01.y + cb * x01.y);
          y11 = make_double2(y11.x + cb * x11.x, y11.y + cb * x11.y);
          // B = Ja^H Y:  row0 = c Y0 - sig Y1, row1 = conj(sig) Y0 + c Y1
          const double2 sac = make_double2(sa.x, -sa.y);
          double2 t0 = cmul_d(sa, y10), t1 = cmul_d(sa, y11);
          double2 b00 = make_double2(ca * y00.x - t0.x, ca * y00.y - t0.y);
          double2 b01 = make_double2(ca * y01.x - t1.x, ca * y01.y - t1.y);
          double2 u0 = cmul_d(sac, y00), u1 = cmul_d(sac, y01);
          double2 b10 = make_double2(u0.x + ca * y10.x, u0.y + ca * y10.y);
          double2 b11 = make_double2(u1.x + ca * y11.x, u1.y + ca * y11.y);
          if (ia == ib) {                    // the pair's own block: diagonal by construction
            b00.y = 0.0;
            b11.y = 0.0;
            b01 = z;
            b10 = z;
          }
          __stcg(A + (int64_t)pa * n + pb, b00);
          if (qb_ok) __stcg(A + (int64_t)pa * n + qb, b01);
          if (qa_ok) __stcg(A + (int64_t)qa * n + pb, b10);
          if (qa_ok && qb_ok) __stcg(A + (int64_t)qa * n + qb, b11);
        } else {
          const int64_t f = e - nblk;
          const int i = (int)(f / half), ib = (int)(f % half);
          int pb = rr_index(ib, r, ne), qb = rr_index(ne - 1 - ib, r, ne);
          if (pb > qb) { const int x = pb; pb = qb; qb = x; }
          if (qb >= n) continue;
          const double cb = __ldcg(rot + 2 * ib).x;
          const double2 sb = __ldcg(rot + 2 * ib + 1), sbc = make_double2(sb.x, -sb.y);
          const double2 v0 = ld2(V + (int64_t)i * n + pb), v1 = ld2(V + (int64_t)i * n + qb);
          const double2 a0 = cmul_d(sbc, v1), a1 = cmul_d(sb, v0);
          __stcg(V + (int64_t)i * n + pb, make_double2(cb * v0.x - a0.x, cb * v0.y - a0.y));
          __stcg(V + (int64_t)i * n + qb, make_double2(a1.x + cb * v1.x, a1.y + cb * v1.y));
        }
      }
      if (!grid_sync(bar, nb, status)) return;
    }
  }
  for (int64_t i = tid; i < n; i += nthr) lam[i] = ld2(A + i * n + i).x;
  if (tid == 0) {
    info[0] = (double)sweep;
    info[1] = sqrt(off / fmax(fro, 1e-300));
    if (!(off <= tol * tol * fro)) flag_error(status, DEV_ERR_NUMERIC);
  }
}

// ---------------------------------------------------------------------------------------
// eigenbasis quantities: rho_k = sum_l conj(V_lk) F_l and (optionally) the energy-weighted
// second moment qd_k = sum_{l,l'} conj(V_lk) Q_ll' V_l'k; one block per k
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tdvp_project(const double2* __restrict__ V,
                                                      const double2* __restrict__ F,
                                                      const double2* __restrict__ Q, int64_t P,
                                                      double2* rho, double* qd) {
  __shared__ double sh[32];
  const int64_t k = blockIdx.x;
  double rr = 0, ri = 0, qq = 0;
  for (int64_t l = threadIdx.x; l < P; l += blockDim.x) {
    const double2 v = V[l * P + k];
    const double2 f = F[l];
    const double2 p = cconjmul_d(v, f);
    rr += p.x;
    ri += p.y;
    if (Q) {
      double2 u = make_double2(0, 0);               // (Q V_k)_l, Q_lm = conj(Q_ml)
      for (int64_t m = 0; m < P; ++m) {
        const double2 x = cconjmul_d(Q[m * P + l], V[m * P + k]);
        u.x += x.x;
        u.y += x.y;
      }
      qq += cconjmul_d(v, u).x;
    }
  }
  rr = block_sum(rr, sh);
  ri = block_sum(ri, sh);
  if (Q) qq = block_sum(qq, sh);
  if (threadIdx.x == 0) {
    rho[k] = make_double2(rr, ri);
    if (qd) qd[k] = qq;
  }
}

// lambda^+ of every eigenvalue (one block): pinv cutoff (hard or soft) times the SNR
// damping; st[0..3] = lambda_1 = max |lambda|, min lambda, number of components with a
// damping factor >= 1/2, smallest SNR (0 when not used)
__global__ void k_tdvp_lamplus(const double* __restrict__ lam, const double2* __restrict__ rho,
                               const double* __restrict__ qd, int64_t P, double eps_pinv,
                               int soft, double eps_snr, double n_eff, double* lamp, double* st) {
  __shared__ double sh[32];
  double m = 0.0, mn = INFINITY;
  for (int64_t k = threadIdx.x; k < P; k += blockDim.x) {
    m = fmax(m, fabs(lam[k]));
    mn = fmin(mn, lam[k]);
  }
  const double lam1 = block_max(m, sh);
  const double lmin = -block_max(-mn, sh);
  double kept = 0.0, snr_min = INFINITY;
  for (int64_t k = threadIdx.x; k < P; k += blockDim.x) {
    const double l = lam[k];
    const double r = lam1 > 0.0 ? fabs(l) / lam1 : 0.0;
    double d;
    if (eps_pinv > 0.0) {
      if (soft) {
        const double x = r > 0.0 ? eps_pinv / r : INFINITY;
        d = 1.0 / (1.0 + x * x * x * x * x * x);
      } else {
        d = r >= eps_pinv ? 1.0 : 0.0;
      }
    } else {
      d = l != 0.0 ? 1.0 : 0.0;
    }
    if (eps_snr > 0.0 && qd) {
      const double a2 = rho[k].x * rho[k].x + rho[k].y * rho[k].y;
      const double var = fmax(qd[k] - a2, 0.0);
      const double snr = var > 0.0 ? sqrt(a2) / sqrt(var / n_eff) : INFINITY;
      snr_min = fmin(snr_min, snr);
      const double x = snr > 0.0 ? eps_snr / snr : INFINITY;
      d = d / (1.0 + x * x * x * x * x * x);
    }
    const double lp = (l != 0.0 && d > 0.0) ? d / l : 0.0;
    lamp[k] = isfinite(lp) ? lp : 0.0;
    kept += d >= 0.5 ? 1.0 : 0.0;
  }
  kept = block_sum(kept, sh);
  const double smin = -block_max(-snr_min, sh);
  if (threadIdx.x == 0) {
    st[0] = lam1;
    st[1] = lmin;
    st[2] = kept;
    st[3] = (eps_snr > 0.0 && qd) ? smin : 0.0;
  }
}

// thetadot_l = -gamma sum_k V_lk lambda^+_k rho_k (thread per l)
__global__ void k_tdvp_thetadot(const double2* __restrict__ V, const double* __restrict__ lamp,
                                const double2* __restrict__ rho, int64_t P, double g_re,
                                double g_im, double2* out, unsigned* status) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= P) return;
  double2 acc = make_double2(0, 0);
  for (int64_t k = 0; k < P; ++k) {
    const double c = lamp[k];
    if (c == 0.0) continue;
    const double2 x = cmul_d(V[l * P + k], rho[k]);
    acc.x = fma(c, x.x, acc.x);
    acc.y = fma(c, x.y, acc.y);
  }
  const double2 g = make_double2(-g_re, -g_im);
  const double2 r = cmul_d(g, acc);
  if (!isfinite(r.x) || !isfinite(r.y)) flag_error(status, DEV_ERR_NUMERIC);
  out[l] = r;
}

// multiplicative diagonal shift S_kk <- (1 + nu) S_kk (section "Diagonal shift")
__global__ void k_shift_diag(double2* S, int64_t P, double nu) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < P) S[k * P + k].x *= (1.0 + nu);
}

// out = y + a k1 + b k2 (complex vectors, real coefficients)
__global__ void k_axpy2(const double2* y, double a, const double2* k1, double b, const double2* k2,
                        int64_t P, double2* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const double2 u = y[i], p = k1[i];
  double2 r = make_double2(fma(a, p.x, u.x), fma(a, p.y, u.y));
  if (k2) {
    const double2 q = k2[i];
    r = make_double2(fma(b, q.x, r.x), fma(b, q.y, r.y));
  }
  out[i] = r;
}

// per-block partials of v^H S v (v = x - y, S Hermitian) (block per 256 rows; thread per row)
__global__ void k_quad_form(const double2* __restrict__ S, const double2* __restrict__ x,
                            const double2* __restrict__ y, int64_t P, double* part) {
  __shared__ double sh[32];
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (l < P) {
    double2 u = make_double2(0, 0);
    for (int64_t m = 0; m < P; ++m) {
      const double2 v = make_double2(x[m].x - y[m].x, x[m].y - y[m].y);
      const double2 p = cconjmul_d(S[m * P + l], v);      // S_lm = conj(S_ml)
      u.x += p.x;
      u.y += p.y;
    }
    const double2 vl = make_double2(x[l].x - y[l].x, x[l].y - y[l].y);
    acc = cconjmul_d(vl, u).x;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
int64_t tdvp_gram_partial_doubles2(int64_t n, int64_t P, int n_sm) {
  const int64_t tiles_1d = (P + kTile - 1) / kTile;
  const int64_t ntiles = tiles_1d * (tiles_1d + 1) / 2;
  const int64_t chunks = tdvp_gram_chunks(n, P, n_sm);
  return chunks * ntiles * kTile * kTile * 2;
}

int64_t tdvp_gram_chunks(int64_t n, int64_t P, int n_sm) {
  const int64_t tiles_1d = (P + kTile - 1) / kTile;
  const int64_t ntiles = tiles_1d * (tiles_1d + 1) / 2;
  int64_t c = std::max<int64_t>(1, (2 * (int64_t)n_sm + ntiles - 1) / ntiles);
  c = std::min<int64_t>(c, std::max<int64_t>(1, n / 512));          // >= 512 samples a chunk
  c = std::min<int64_t>(c, std::max<int64_t>(1, (int64_t)(64 << 20) / (ntiles * 1024 * 2)));
  return c;
}

cudaError_t launch_enum_states(int8_t* spins, int N, int64_t n, cudaStream_t st) {
  const int64_t tot = n * N;
  k_enum_states<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(spins, N, n);
  return cudaGetLastError();
}

cudaError_t launch_born_weights(const float2* lp, int64_t n, double* w, unsigned* status,
                                cudaStream_t st) {
  k_born_weights<<<1, 1024, 0, st>>>(lp, n, w, status);
  return cudaGetLastError();
}

cudaError_t launch_normalize_weights(const double* w_in, int64_t n, double* w_out,
                                     unsigned* status, cudaStream_t st, double* sums) {
  k_normalize_weights<<<1, 1024, 0, st>>>(w_in, n, w_out, status, sums);
  return cudaGetLastError();
}

cudaError_t tdvp_moments(const int8_t* spins, const float2* T, const float2* E, const double* w,
                         const float2* osc, int64_t n, int N, int M, TdvpWork& tw,
                         cudaStream_t st, const float* Od, int64_t Pd) {
  const int64_t P = Od ? Pd : (int64_t)N + M + (int64_t)N * M;
  k_tdvp_energy<<<1, 1024, 0, st>>>(E, w, n, tw.estats, tw.status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t kb = (P + 255) / 256;
  int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((2 * tw.n_sm + kb - 1) / kb, n / 256));
  chunks = std::min<int64_t>(chunks, tw.mom_part_cap / (2 * P));
  chunks = std::max<int64_t>(chunks, 1);
  const int64_t chunk = (n + chunks - 1) / chunks;
  chunks = (n + chunk - 1) / chunk;
  k_tdvp_moments<<<dim3((unsigned)kb, (unsigned)chunks), 256, 0, st>>>(
      spins, T, E, w, osc, Od, tw.estats, n, N, M, P, chunk, tw.mom_part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_tdvp_moments_reduce<<<(unsigned)kb, 256, 0, st>>>(tw.mom_part, (int)chunks, P, tw.meanO, tw.F);
  return cudaGetLastError();
}

cudaError_t tdvp_gram(const int8_t* spins, const float2* T, const float2* E, const double* w,
                      const float2* osc, int64_t n, int N, int M, TdvpWork& tw,
                      cudaStream_t st, const float* Od, int64_t Pd) {
  const int64_t P = Od ? Pd : (int64_t)N + M + (int64_t)N * M;
  const int64_t tiles_1d = (P + kTile - 1) / kTile;
  const int64_t ntiles = tiles_1d * (tiles_1d + 1) / 2;
  int64_t chunks = tdvp_gram_chunks(n, P, tw.n_sm);
  while (chunks > 1 && chunks * ntiles * kTile * kTile * 2 > tw.gram_part_cap) --chunks;
  if (chunks * ntiles * kTile * kTile * 2 > tw.gram_part_cap) return cudaErrorInvalidValue;
  const int64_t chunk = (n + chunks - 1) / chunks;
  chunks = (n + chunk - 1) / chunk;
  k_tdvp_gram<<<dim3((unsigned)ntiles, (unsigned)chunks), 256, 0, st>>>(
      spins, T, E, w, osc, Od, tw.estats, tw.meanO, n, N, M, P, chunk, ntiles, tw.gram_part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tdvp_gram_reduce<<<(unsigned)ntiles, kTile * kTile, 0, st>>>(tw.gram_part, (int)chunks, ntiles,
                                                               P, tw.S, tw.Q);
  return cudaGetLastError();
}

cudaError_t tdvp_eig(TdvpWork& tw, int64_t P, int max_sweeps, double tol, cudaStream_t st) {
  // the work matrix A = S (copied; S itself is kept for the Fisher norm)
  cudaError_t e = cudaMemcpyAsync(tw.A, tw.S, sizeof(double2) * P * P, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(tw.bar, 0, 4 * sizeof(unsigned), st)) != cudaSuccess) return e;
  int n = (int)P, ne = n + (n & 1);
  const int64_t items = std::max<int64_t>((int64_t)(ne / 2) * (ne / 2) + (int64_t)n * (ne / 2),
                                          (int64_t)n * n);
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_eig, 256, 0)) != cudaSuccess)
    return e;
  int grid = (int)std::min<int64_t>((items + 255) / 256, (int64_t)per_sm * tw.n_sm);
  grid = std::max(1, std::min(grid, tw.red_cap));
  void* args[] = {&tw.A, &tw.V, &n, &ne, &tw.lam, &tw.rot, &tw.bar, &tw.red, &tw.status,
                  &max_sweeps, &tol, &tw.info};
  return cudaLaunchCooperativeKernel((const void*)k_jacobi_eig, dim3(grid), dim3(256), args, 0, st);
}

cudaError_t tdvp_solve(TdvpWork& tw, int64_t P, bool snr, double eps_pinv, int soft,
                       double eps_snr, double n_eff, double g_re, double g_im, double2* out,
                       cudaStream_t st) {
  k_tdvp_project<<<(unsigned)P, 256, 0, st>>>(tw.V, tw.F, snr ? tw.Q : nullptr, P, tw.rho,
                                              snr ? tw.qd : nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_tdvp_lamplus<<<1, 1024, 0, st>>>(tw.lam, tw.rho, snr ? tw.qd : nullptr, P, eps_pinv, soft,
                                     snr ? eps_snr : 0.0, n_eff, tw.lamp, tw.lstats);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_tdvp_thetadot<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(tw.V, tw.lamp, tw.rho, P, g_re, g_im,
                                                               out, tw.status);
  return cudaGetLastError();
}

cudaError_t tdvp_shift(TdvpWork& tw, int64_t P, double nu, cudaStream_t st) {
  k_shift_diag<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(tw.S, P, nu);
  return cudaGetLastError();
}

cudaError_t launch_axpy2(const double2* y, double a, const double2* k1, double b, const double2* k2,
                         int64_t P, double2* out, cudaStream_t st) {
  k_axpy2<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(y, a, k1, b, k2, P, out);
  return cudaGetLastError();
}

cudaError_t launch_quad_form(const double2* S, const double2* x, const double2* y, int64_t P,
                             double* part, int* nparts, cudaStream_t st) {
  *nparts = (int)((P + 255) / 256);
  k_quad_form<<<(unsigned)*nparts, 256, 0, st>>>(S, x, y, P, part);
  return cudaGetLastError();
}

}  // namespace vmc
