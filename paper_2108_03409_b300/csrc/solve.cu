// solve.cu -- regularised solve of S~ x = F (section "Diagonal shift"; Algorithm 1,
// solve_TDVP_equation) by a blocked right-looking complex Cholesky factorisation
// S~ = L L^H, in FP64, or in FP32 followed by FP64 iterative refinement against the
// FP64 S~.  Diagonal blocks of L are inverted once so that the panel solve and the
// triangular solves become small matrix products.
#include <type_traits>

#include "tc_ptx.cuh"
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

// Factor the 64 x 64 diagonal block (rows/cols k0..k0+kw) and store its inverse; one CTA
// of 256 threads, the block in shared memory (identity padding beyond kw, masked on output).
//  * Factorisation in four 16-column panels.  Within a panel warp w keeps the columns
//    c0 + 2w, c0 + 2w + 1 in registers, lane l rows c0 + l and c0 + l + 32 of both; per
//    column pair the owner warp resolves the 2x2 pivot block (two pivot shuffles and one
//    for L[c+1][c]; every lane scales and updates its own rows), publishes both columns
//    (double-buffered), one barrier, then the later warps apply the rank-2 update.  After
//    the panel the trailing triangle gets one rank-16 update.
//  * The outer loops stay rolled: inside the panel kernel the code is fetched while the
//    other CTAs stream the panel through L2, and a compact loop body runs faster there
//    than the fully unrolled one (which wins only on an idle GPU).
//  * Inverse: the four 16 x 16 diagonal blocks are inverted at once (forward substitution
//    on the identity, one warp each, a column per lane), then the off-diagonal 16-blocks by
//    levels, X_ij = -D_i sum_{k=j}^{i-1} L_ik X_kj (D_i = diagonal inverse).
constexpr int POTRF_THREADS = 256;
constexpr int PLD = NB + 1;

// Pivot root: l = sqrt(d), il = 1 / l.  In FP32 from the hardware reciprocal square root
// (the factor only preconditions the FP64-accurate refinement, and l il = 1 to rounding);
// in FP64 correctly rounded.
__device__ __forceinline__ void pivot_root(float d, float* l, float* il) {
  *il = rsqrtf(d);
  *l = d * *il;
}
__device__ __forceinline__ void pivot_root(double d, double* l, double* il) {
  *l = sqrt(d);
  *il = 1.0 / *l;
}

// (Global loads bypass L1 (ld.global.cg): inside the cooperative panel kernel the block
// may have been written by other CTAs since this SM last cached it.)
// Shared-memory layout of the diagonal-block factorisation (psm: potrf_smem bytes)
template <typename C> struct PotrfSmem {
  C* a;    // [64][PLD]: A -> L
  C* li;   // [64][PLD]: Linv
  C* tt;   // [64][PLD]: products of the inverse
  C* cb;   // [2][2][64]: published column pair / row
  typename RealOf<C>::T* dg;  // [64]: 1 / L_cc
  __device__ explicit PotrfSmem(unsigned char* psm) {
    a = reinterpret_cast<C*>(psm);
    li = a + NB * PLD;
    tt = li + NB * PLD;
    cb = tt + NB * PLD;
    dg = reinterpret_cast<typename RealOf<C>::T*>(cb + 4 * NB);
  }
};

// the lower triangle of the diagonal block (identity padding beyond kw) into a
template <typename C>
__device__ void potrf_load(const C* __restrict__ A, int64_t P, int64_t k0, int kw, C* a) {
  // all of a thread's loads are issued before any shared-memory store
  constexpr int PER = NB * NB / POTRF_THREADS;
  C v[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = threadIdx.x + POTRF_THREADS * u, r = e >> 6, c = e & 63;
    v[u] = (r < kw && c <= r) ? __ldcg(&A[(k0 + r) * P + k0 + c])
                              : mk<C>((r == c && r >= kw) ? 1.0 : 0.0, 0.0);
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = threadIdx.x + POTRF_THREADS * u, r = e >> 6, c = e & 63;
    a[r * PLD + c] = v[u];
  }
}

// L and Linv back to A and Dinv
template <typename C>
__device__ void potrf_store(C* __restrict__ A, int64_t P, int64_t k0, int kw,
                            C* __restrict__ Dinv, const C* a, const C* li) {
  for (int e = threadIdx.x; e < NB * NB; e += POTRF_THREADS) {
    const int r = e >> 6, c = e & 63;
    if (r < kw && c <= r) A[(k0 + r) * P + k0 + c] = a[r * PLD + c];
    Dinv[e] = (r < kw && c < kw && c <= r) ? li[r * PLD + c] : mk<C>(0.0, 0.0);
  }
}

// Factor the block held in sm.a (lower triangle, identity padding) in place and form its
// inverse in sm.li; returns with a barrier passed after the last shared-memory write.
template <typename C>
__device__ void potrf_core(unsigned* status, const PotrfSmem<C>& sm) {
  typedef typename RealOf<C>::T R;
  C* a = sm.a;
  C* li = sm.li;
  C* tt = sm.tt;
  C* cb = sm.cb;
  R* dg = sm.dg;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += POTRF_THREADS) li[(e >> 6) * PLD + (e & 63)] = mk<C>(0.0, 0.0);
  __syncthreads();
  bool bad = false;
  const int warp = tid >> 5, lane = tid & 31;
  int pb = 0;
#pragma unroll 1
  for (int pp = 0; pp < 4; ++pp) {
    const int c0 = 16 * pp;
    // warp w owns the panel columns c0 + 2w + q (q = 0, 1); lane l the rows c0 + l + 32h
    C e[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int r = c0 + lane + 32 * h;
        e[h][q] = (r < NB) ? a[r * PLD + c0 + 2 * warp + q] : mk<C>(0.0, 0.0);
      }
    // column pairs (c, c+1) = (c0 + 2w, c0 + 2w + 1): the owner warp resolves the 2x2 pivot
    // block (each lane scales its own rows of column c and updates its own rows of column
    // c+1; three shuffles), publishes both columns, one barrier, then the later warps apply
    // the rank-2 update to their columns
#pragma unroll 1
    for (int w = 0; w < 8; ++w) {
      const int c = c0 + 2 * w;
      C* cbA = cb + pb * 2 * NB;                     // column c
      C* cbB = cbA + NB;                             // column c + 1
      if (warp == w) {
        R d0 = __shfl_sync(0xffffffffu, e[0][0].x, 2 * w);      // (c, c): row c0 + 2w
        if (!(d0 > (R)0) || !isfinite(d0)) { bad |= (lane == 0); d0 = (R)1; }
        R l0, il0;
        pivot_root(d0, &l0, &il0);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = c0 + lane + 32 * h;
          if (r > c) {
            e[h][0].x *= il0;
            e[h][0].y *= il0;
          } else if (r == c) {
            e[h][0] = mk<C>((double)l0, 0.0);
          }
        }
        C lw;                                                    // L[c+1][c]
        lw.x = __shfl_sync(0xffffffffu, e[0][0].x, 2 * w + 1);
        lw.y = __shfl_sync(0xffffffffu, e[0][0].y, 2 * w + 1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = c0 + lane + 32 * h;
          if (r > c) {
            e[h][1].x -= e[h][0].x * lw.x + e[h][0].y * lw.y;
            e[h][1].y -= e[h][0].y * lw.x - e[h][0].x * lw.y;
          }
        }
        R d1 = __shfl_sync(0xffffffffu, e[0][1].x, 2 * w + 1);  // (c+1, c+1)
        if (!(d1 > (R)0) || !isfinite(d1)) { bad |= (lane == 0); d1 = (R)1; }
        R l1, il1;
        pivot_root(d1, &l1, &il1);
        if (lane == 0) {
          dg[c] = il0;
          dg[c + 1] = il1;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = c0 + lane + 32 * h;
          if (r > c + 1 && r < NB) {
            e[h][1].x *= il1;
            e[h][1].y *= il1;
            cbB[r] = e[h][1];
          } else if (r == c + 1) {
            e[h][1] = mk<C>((double)l1, 0.0);
          }
          if (r > c && r < NB) cbA[r] = e[h][0];
        }
      }
      __syncthreads();
      if (warp > w) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int cc = c0 + 2 * warp + q;
          const C la = cbA[cc], lb = cbB[cc];                    // L[cc][c], L[cc][c+1]
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = c0 + lane + 32 * h;
            if (r >= cc && r < NB) {
              const C ra = cbA[r], rb = cbB[r];
              e[h][q].x -= ra.x * la.x + ra.y * la.y + rb.x * lb.x + rb.y * lb.y;
              e[h][q].y -= ra.y * la.x - ra.x * la.y + rb.y * lb.x - rb.x * lb.y;
            }
          }
        }
      }
      pb ^= 1;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int r = c0 + lane + 32 * h;
        if (r < NB) a[r * PLD + c0 + 2 * warp + q] = e[h][q];
      }
    __syncthreads();
    if (pp < 3) {
      // trailing rank-16 update of rows/cols >= c0 + 16 (lower triangle)
      const int t0 = c0 + 16;
      const int ty = tid & 15, tx = tid >> 4;
#pragma unroll 1
      for (int p = 0; p < 4; ++p) {
        const int r = ty + 16 * p;
        if (r < t0) continue;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
          const int cc = tx + 16 * q;
          if (cc < t0 || cc > r) continue;
          C acc = mk<C>(0.0, 0.0);
#pragma unroll 4
          for (int m = 0; m < 16; ++m) cfmac(acc, a[r * PLD + c0 + m], a[cc * PLD + c0 + m]);
          a[r * PLD + cc].x -= acc.x;
          a[r * PLD + cc].y -= acc.y;
        }
      }
      __syncthreads();
    }
  }
  if (bad) flag_error(status, DEV_ERR_NUMERIC);
  // ---- inverse: 16 x 16 diagonal blocks, one warp each; lane (j, h) forms column j of
  // the block's inverse by forward substitution (both row halves form the whole column,
  // each stores its own rows); no barrier ----
  if (warp < 4) {
    const int b0 = 16 * warp, j = lane & 15, h = lane >> 4;
    C x[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) x[m] = mk<C>((m == j) ? 1.0 : 0.0, 0.0);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const R il = dg[b0 + k];
      x[k].x *= il;
      x[k].y *= il;
#pragma unroll
      for (int m = k + 1; m < 16; ++m) {
        const C lmk = a[(b0 + m) * PLD + b0 + k];
        x[m].x -= lmk.x * x[k].x - lmk.y * x[k].y;
        x[m].y -= lmk.x * x[k].y + lmk.y * x[k].x;
      }
    }
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if ((m >> 3) == h && m >= j) li[(b0 + m) * PLD + b0 + j] = x[m];
  }
  __syncthreads();
  // ---- off-diagonal 16-blocks by levels d = i - j (each thread holds 4 - d entries of a
  // level; the levels and entry counts are compile-time, so a thread's entries interleave) ----
#pragma unroll 1
  for (int d = 1; d < 4; ++d) {
    constexpr int kMaxNb = 3;
    const int nb = 4 - d;                          // blocks (j + d, j), j < nb
    // T_ij = sum_{k=j}^{i-1} L_ik X_kj, into tt at block (i, j)
    C acc[kMaxNb];
#pragma unroll
    for (int u = 0; u < kMaxNb; ++u) {
      acc[u] = mk<C>(0.0, 0.0);
      if (u < nb) {
        const int e = tid + POTRF_THREADS * u;
        const int j = e >> 8, i = j + d, r = (e >> 4) & 15, c = e & 15;
#pragma unroll 1
        for (int k2 = 0; k2 < d; ++k2) {
          const int k = j + k2;
#pragma unroll 4
          for (int m = 0; m < 16; ++m)
            cfma(acc[u], a[(16 * i + r) * PLD + 16 * k + m], li[(16 * k + m) * PLD + 16 * j + c]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kMaxNb; ++u)
      if (u < nb) {
        const int e = tid + POTRF_THREADS * u;
        const int j = e >> 8, i = j + d, r = (e >> 4) & 15, c = e & 15;
        tt[(16 * i + r) * PLD + 16 * j + c] = acc[u];
      }
    __syncthreads();
    // X_ij = -D_i T_ij
#pragma unroll
    for (int u = 0; u < kMaxNb; ++u) {
      acc[u] = mk<C>(0.0, 0.0);
      if (u < nb) {
        const int e = tid + POTRF_THREADS * u;
        const int j = e >> 8, i = j + d, r = (e >> 4) & 15, c = e & 15;
#pragma unroll 4
        for (int m = 0; m < 16; ++m)
          cfma(acc[u], li[(16 * i + r) * PLD + 16 * i + m], tt[(16 * i + m) * PLD + 16 * j + c]);
      }
    }
#pragma unroll
    for (int u = 0; u < kMaxNb; ++u)
      if (u < nb) {
        const int e = tid + POTRF_THREADS * u;
        const int j = e >> 8, i = j + d, r = (e >> 4) & 15, c = e & 15;
        li[(16 * i + r) * PLD + 16 * j + c] = mk<C>(-(double)acc[u].x, -(double)acc[u].y);
      }
    __syncthreads();
  }
}

template <typename C>
__device__ void potrf_body(C* __restrict__ A, int64_t P, int64_t k0, int kw,
                           C* __restrict__ Dinv, unsigned* status, unsigned char* psm) {
  const PotrfSmem<C> sm(psm);
  potrf_load<C>(A, P, k0, kw, sm.a);
  potrf_core<C>(status, sm);
  potrf_store<C>(A, P, k0, kw, Dinv, sm.a, sm.li);
}

template <typename C>
__global__ void __launch_bounds__(POTRF_THREADS) k_potrf_diag(C* __restrict__ A, int64_t P,
                                                              int64_t k0, int kw,
                                                              C* __restrict__ Dinv,
                                                              unsigned* status) {
  extern __shared__ unsigned char psm[];
  potrf_body<C>(A, P, k0, kw, Dinv, status, psm);
}

// Where the row solves of a tensor-core panel also write their results: rows r0 .. r0+n-1
// (the rows below the panel) become rows 2(row - r0) (real) and 2(row - r0) + 1 (imaginary)
// of the BF16 hi/lo operand planes [rows_pad][K] of the panel's Schur update, column m.
// hi == nullptr: no operand output.
struct XOut {
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  int64_t r0, n;
  int K, m0;                                     // m0: the panel column of the block's column 0
};

// The solved rows r0 .. r0 + nrow - 1, staged in st (row stride NB + 1, columns 0 .. kw-1):
// those below the panel go into the operand planes, 16 bytes (eight columns of one real
// row, hi or lo) per store.  Work item (row, component, eight-column chunk).
__device__ __forceinline__ void x_store_rows(const XOut& xo, const float2* st, int64_t r0,
                                             int nrow, int kw) {
  if (xo.hi == nullptr) return;
  for (int it = threadIdx.x; it < nrow * 16; it += blockDim.x) {
    const int r = it >> 4, comp = (it >> 3) & 1, ch = it & 7;
    const int64_t row = r0 + r;
    if (row < xo.r0 || row - xo.r0 >= xo.n || 8 * ch >= kw) continue;
    const float2* src = st + r * (NB + 1) + 8 * ch;
    const int64_t off = (2 * (row - xo.r0) + comp) * xo.K + xo.m0 + 8 * ch;
    if (8 * ch + 8 <= kw) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 a = src[2 * e], b = src[2 * e + 1];
        tc::split_pair(comp ? a.y : a.x, comp ? b.y : b.x, h[e], l[e]);
      }
      *reinterpret_cast<uint4*>(xo.hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(xo.lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    } else {
      for (int e = 0; 8 * ch + e < kw; ++e) {
        const float x = comp ? src[e].y : src[e].x;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        xo.hi[off + e] = h;
        xo.lo[off + e] = __float2bfloat16_rn(x - __bfloat162float(h));
      }
    }
  }
}

// Panel: X = B L_kk^{-H}, X[r][c] = sum_m B[r][m] conj(Linv[c][m]) (Linv is zero above its
// diagonal) for the rows below the diagonal block; 64 rows per block, written over the
// panel of A.  Thread (ty, tx) accumulates the 4 x 4 outputs (ty + 16a, tx + 16b).
template <typename C>
__device__ void trsm_body(C* __restrict__ A, int64_t P, int64_t k0, int kw,
                          const C* __restrict__ Dinv, int64_t r0, unsigned char* tsm,
                          const XOut& xo = XOut{nullptr, nullptr, 0, 0, 0, 0}) {
  C* Bt = reinterpret_cast<C*>(tsm);           // [NB (m)][NB+1 (r)]
  C* Lt = Bt + NB * (NB + 1);                  // [NB (m)][NB+1 (c)]
  const int tid = threadIdx.x;
  {
    constexpr int PER = NB * NB / 256;
    C bv[PER], lv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u, rr = e / NB, m = e % NB;
      const int64_t row = r0 + rr;
      bv[u] = (row < P && m < kw) ? __ldcg(&A[row * P + k0 + m]) : mk<C>(0.0, 0.0);
      lv[u] = __ldcg(&Dinv[e]);                  // e = c * NB + m with c = rr
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u, rr = e / NB, m = e % NB;
      Bt[m * (NB + 1) + rr] = bv[u];
      Lt[m * (NB + 1) + rr] = lv[u];
    }
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<C>(0.0, 0.0);
  // Linv is lower triangular: columns m of block jb reach only the column blocks j >= jb
#pragma unroll
  for (int jb = 0; jb < 4; ++jb) {
    const int mend = min(kw, 16 * jb + 16);
    for (int m = 16 * jb; m < mend; ++m) {
      C br[4], lc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) br[i] = Bt[m * (NB + 1) + ty + 16 * i];
#pragma unroll
      for (int j = jb; j < 4; ++j) lc[j] = Lt[m * (NB + 1) + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = jb; j < 4; ++j) cfmac(acc[i][j], br[i], lc[j]);
    }
  }
  // stage X (over B^T, once every thread is done reading it), then store it coalesced
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) Bt[(ty + 16 * i) * (NB + 1) + tx + 16 * j] = acc[i][j];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NB * NB / 256; ++u) {
    const int e = tid + 256 * u, r = e >> 6, c = e & 63;
    const int64_t row = r0 + r;
    if (row < P && c < kw) A[row * P + k0 + c] = Bt[r * (NB + 1) + c];
  }
  if constexpr (std::is_same<C, float2>::value) x_store_rows(xo, Bt, r0, NB, kw);
}

template <typename C>
__global__ void __launch_bounds__(256) k_trsm_inv(C* __restrict__ A, int64_t P, int64_t k0,
                                                  int kw, const C* __restrict__ Dinv) {
  extern __shared__ unsigned char tsm[];
  trsm_body<C>(A, P, k0, kw, Dinv, k0 + kw + (int64_t)blockIdx.x * NB, tsm);
}

// Trailing update of one lower 64x64 tile (rows r0.., columns c0..):
// A[r][c] -= sum_m X[r][m] conj(X[c][m]) for c <= r, X = the panel A[.][k0 .. k0+kw).
// The tile's current values are fetched before the products so that their latency
// overlaps the arithmetic.
template <typename C>
__device__ void herk_tile_body(C* __restrict__ A, int64_t P, int64_t k0, int kw, int64_t r0,
                               int64_t c0, unsigned char* hsm) {
  C* Xr = reinterpret_cast<C*>(hsm);           // [NB (m)][NB+1 (row)]
  C* Xc = Xr + NB * (NB + 1);                  // [NB (m)][NB+1 (col)]
  const int tid = threadIdx.x;
  {
    constexpr int PER = NB * NB / 256;
    C rv[PER], cv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u, rr = e / NB, m = e % NB;
      const int64_t row = r0 + rr, col = c0 + rr;
      rv[u] = (row < P && m < kw) ? __ldcg(&A[row * P + k0 + m]) : mk<C>(0.0, 0.0);
      cv[u] = (col < P && m < kw) ? __ldcg(&A[col * P + k0 + m]) : mk<C>(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u, rr = e / NB, m = e % NB;
      Xr[m * (NB + 1) + rr] = rv[u];
      Xc[m * (NB + 1) + rr] = cv[u];
    }
  }
  const int tx = tid & 15, ty = tid >> 4;
  C cur[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t row = r0 + ty + 16 * a, col = c0 + tx + 16 * b;
      cur[a][b] = (row < P && col < P && col <= row) ? __ldcg(&A[row * P + col]) : mk<C>(0.0, 0.0);
    }
  __syncthreads();
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
        C v = cur[a][b];
        v.x -= acc[a][b].x;
        v.y -= acc[a][b].y;
        A[row * P + col] = v;
      }
    }
  }
}

// tile t of the trapezoid below k1 = k0 + kw restricted to nct tile columns, column by
// column (column tn holds tiles tm = tn .. nt-1)
__device__ __forceinline__ void trapezoid_tile(int64_t t, int64_t nt, int64_t* tm, int64_t* tn) {
  int64_t u = t, c = 0;
  while (u >= nt - c) { u -= nt - c; ++c; }
  *tn = c;
  *tm = c + u;
}

// Trailing update on lower 64x64 tiles for columns c < col_end (col_end >= P: the whole
// trailing matrix; otherwise a trapezoid of a few tile columns, used inside a panel).
template <typename C>
__global__ void __launch_bounds__(256) k_herk(C* __restrict__ A, int64_t P, int64_t k0, int kw,
                                              int64_t col_end) {
  extern __shared__ unsigned char hsm[];
  const int64_t k1 = k0 + kw;
  const int64_t t = blockIdx.x;
  int64_t tm, tn;
  if (col_end >= P) {                        // lower-triangular tile enumeration
    tm = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
    while (tm * (tm + 1) / 2 > t) --tm;
    tn = t - tm * (tm + 1) / 2;
  } else {
    trapezoid_tile(t, (P - k1 + NB - 1) / NB, &tm, &tn);
  }
  herk_tile_body<C>(A, P, k0, kw, k1 + tm * NB, k1 + tn * NB, hsm);
}

// ---------------------------------------------------------------------------------------
// Whole triangular solves in one cooperative launch: the block steps of the forward
// (L y = b) and backward (L^H x = y) substitutions are separated by a grid barrier.  The
// barrier is a counter plus a generation word in global memory; every wait is bounded
// (iteration and clock limits) and an expired wait sets DEV_ERR_TIMEOUT and an abort word
// that makes every block leave the loop.  The right-hand-side vectors are read and written
// with L2-only accesses (ld/st.global.cg): rows move between blocks from step to step, so
// an L1 copy from an earlier step could be stale.
// ---------------------------------------------------------------------------------------
// Bounded waits on a counter in global memory: iteration and clock limits; an expired wait
// sets DEV_ERR_TIMEOUT and the abort word, which every other wait also checks.
__device__ __forceinline__ bool wait_at_least(const unsigned* word, unsigned target,
                                              unsigned* abort_word, unsigned* status) {
  volatile const unsigned* vw = word;
  volatile unsigned* vab = abort_word;
  const long long t0 = clock64();
  unsigned it = 0;
  while (*vw < target) {
    if (*vab) return false;
    if ((++it & 1023u) == 0 && clock64() - t0 > 2000000000ll) {
      atomicExch(abort_word, 1u);
      flag_error(status, DEV_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// CTA-wide: thread 0 waits, the verdict is shared; a fence makes the awaited data visible.
// Barriers on both sides keep the shared verdict from being overwritten by the next call
// before every thread has read it.
__device__ __forceinline__ bool cta_wait(const unsigned* word, unsigned target,
                                         unsigned* abort_word, unsigned* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = wait_at_least(word, target, abort_word, status) ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  const bool r = ok != 0;
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------------------
// In-panel trailing update on the tensor cores: the other CTAs' tiles of a panel step,
//   A[r][c] -= sum_m X[r][m] conj(X[c][m]),  X = the step's 64 solved columns,
// as one real product per 64 x 64 tile.  The 64 rows of X of a tile row (or column) become
// a 128 x 64 BF16 operand, real row 2 rho = Re X[rho], 2 rho + 1 = Im X[rho], split into
// hi + lo (three products hi.hi^T + hi.lo^T + lo.hi^T accumulate in FP32 in tensor memory,
// as in the Schur updates between panels); the 2 x 2 blocks of the 128 x 128 product fold
// to the complex tile.  A CTA takes whole tile rows: the row operand is formed once, the
// column operands per tile; the operands are written into shared memory in the 128-byte
// swizzled K-major layout the MMA descriptors name.  One thread issues the products and
// commits them to an mbarrier; the wait is bounded.
// ---------------------------------------------------------------------------------------
namespace ptc {
constexpr int OP = 128 * 128;                    // one operand plane: 128 rows x 128 bytes
constexpr int A_HI = 0, A_LO = OP, B_HI = 2 * OP, B_LO = 3 * OP, STG = 4 * OP;
constexpr int STG_LD = NB + 1;                   // staging row stride (float2)
constexpr size_t SMEM = 4 * OP + (size_t)NB * STG_LD * sizeof(float2);
constexpr int TMEM_COLS = 128;                   // one 128 x 128 FP32 accumulator
}  // namespace ptc

// rows row0 .. row0 + 63 of the block columns k0 .. k0 + kw of A (zero beyond P and kw), 16
// entries per thread, coalesced along rows; ptc_put stages them into stg
__device__ __forceinline__ void ptc_load(const float2* __restrict__ A, int64_t P, int64_t k0,
                                         int kw, int64_t row0, float2 (&v)[NB * NB / 256]) {
#pragma unroll
  for (int u = 0; u < NB * NB / 256; ++u) {
    const int e = threadIdx.x + 256 * u, rho = e >> 6, m = e & 63;
    const int64_t row = row0 + rho;
    v[u] = (row < P && m < kw) ? __ldcg(&A[row * P + k0 + m]) : make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ void ptc_put(const float2 (&v)[NB * NB / 256], float2* stg) {
#pragma unroll
  for (int u = 0; u < NB * NB / 256; ++u) {
    const int e = threadIdx.x + 256 * u;
    stg[(e >> 6) * ptc::STG_LD + (e & 63)] = v[u];
  }
}

// the staged 64 x 64 complex block as the swizzled BF16 hi/lo operand planes; work item
// (rho, ch) packs columns 8 ch .. 8 ch + 7 of row rho into one 16-byte chunk of each of
// the real rows 2 rho (Re) and 2 rho + 1 (Im) of both planes
__device__ __forceinline__ void ptc_pack(const float2* stg, uint8_t* hi, uint8_t* lo) {
  for (int it = threadIdx.x; it < NB * 8; it += 256) {
    const int rho = it >> 3, ch = it & 7;
    const float2* src = stg + rho * ptc::STG_LD + 8 * ch;
    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 a = src[2 * e], b = src[2 * e + 1];
      tc::split_pair(a.x, b.x, rh[e], rl[e]);
      tc::split_pair(a.y, b.y, ih[e], il[e]);
    }
    const uint32_t o0 = tc::sw128_offset(2 * rho, ch), o1 = tc::sw128_offset(2 * rho + 1, ch);
    *reinterpret_cast<uint4*>(hi + o0) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
    *reinterpret_cast<uint4*>(lo + o0) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<uint4*>(hi + o1) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
    *reinterpret_cast<uint4*>(lo + o1) = make_uint4(il[0], il[1], il[2], il[3]);
  }
  tc::fence_proxy_async_smem();                  // generic writes -> the MMA's async reads
}

// Row block g (rows r0 ..) of step k against the panel's column blocks c = c_lo .. c_hi
// (columns p0 + 64 c ..; c_hi <= g, tile (g, g) lower only).  Before the column operand of
// block c != g is formed, the CTA waits (bounded) until xready[c] reaches 1 (nchain for
// block c_lo, which the chain CTAs solve in slabs): the step's solved rows of block c are
// in A.  sm: 1024-byte aligned, ptc::SMEM bytes.  Returns
// false if a wait expired (DEV_ERR_TIMEOUT recorded, the abort word set).
__device__ __noinline__ bool herk_row_tc(float2* __restrict__ A, int64_t P, int64_t k0, int kw,
                                         int64_t p0, int g, int c_lo, int c_hi,
                                         const unsigned* xready, unsigned nchain, uint8_t* sm,
                                         uint32_t tmem,
                                         uint32_t mbar, uint32_t* phase, volatile int* tc_abort,
                                         int* issued, unsigned* abort_word, unsigned* status) {
  using namespace ptc;
  float2* stg = reinterpret_cast<float2*>(sm + STG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = p0 + (int64_t)g * NB;
  if (c_lo > c_hi) return true;
  float2 v[NB * NB / 256];
  ptc_load(A, P, k0, kw, r0, v);
  __syncthreads();                               // the previous user of the buffers is done
  ptc_put(v, stg);
  __syncthreads();
  ptc_pack(stg, sm + A_HI, sm + A_LO);
  // the column operand's rows are loaded one tile ahead (during the previous products)
  if (c_lo != g) {
    if (!cta_wait(&xready[c_lo], nchain, abort_word, status)) return false;
    ptc_load(A, P, k0, kw, p0 + (int64_t)c_lo * NB, v);
  }
  for (int c = c_lo; c <= c_hi; ++c) {
    const int64_t c0 = p0 + (int64_t)c * NB;
    const bool diag = c == g;
    if (!diag) {
      __syncthreads();                           // stg: the previous tile's update read it
      ptc_put(v, stg);
      __syncthreads();
      ptc_pack(stg, sm + B_HI, sm + B_LO);
    }
    // the tile's current values, fetched before the products complete
    float2 cur[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, rho = e >> 6, q = e & 63;
      const int64_t row = r0 + rho, col = c0 + q;
      cur[u] = (row < P && col < P && (!diag || q <= rho)) ? __ldcg(&A[row * P + col])
                                                           : make_float2(0.f, 0.f);
    }
    tc::fence_before();
    __syncthreads();                             // operands written; accumulator drained
    if (tid == 0) {
      tc::fence_after();
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 128);
      const uint64_t ah = tc::smem_desc_sw128(tc::smem_u32(sm + A_HI));
      const uint64_t al = tc::smem_desc_sw128(tc::smem_u32(sm + A_LO));
      const uint64_t bh = tc::smem_desc_sw128(tc::smem_u32(sm + (diag ? A_HI : B_HI)));
      const uint64_t bl = tc::smem_desc_sw128(tc::smem_u32(sm + (diag ? A_LO : B_LO)));
#pragma unroll
      for (int kk = 0; kk < NB / 16; ++kk) {
        const uint64_t o = (uint64_t)(kk * 32) >> 4;   // 16 BF16 along K
        tc::mma_bf16(tmem, ah + o, bh + o, idesc, kk > 0 ? 1u : 0u);
        tc::mma_bf16(tmem, ah + o, bl + o, idesc, 1u);
        tc::mma_bf16(tmem, al + o, bh + o, idesc, 1u);
      }
      tc::mma_commit(mbar);
      *issued = 1;
    }
    if (c + 1 <= c_hi && c + 1 != g) {           // the next column operand, during the products
      if (!cta_wait(&xready[c + 1], 1u, abort_word, status)) {
        // the products in flight finish before the caller frees the tensor memory
        *tc_abort = 1;
        return false;
      }
      ptc_load(A, P, k0, kw, c0 + NB, v);
    }
    const bool okw = tc::warp_wait(mbar, *phase, tc_abort, lane);
    *phase ^= 1u;
    if (!__syncthreads_and(okw ? 1 : 0)) {
      if (tid == 0) {
        atomicExch(abort_word, 1u);
        flag_error(status, DEV_ERR_TIMEOUT);
      }
      return false;
    }
    tc::fence_after();
    // fold: warp w reads TMEM lanes 32 (w % 4) .. (real rows) and columns 64 (w / 4) ..;
    // row pairs (2 rho, 2 rho + 1) sit in adjacent lanes.  The even row stages the even
    // column pairs, the odd row the odd ones.
    const int qd = warp & 3, hs = warp >> 2;
    const int i = 32 * qd + lane, rho = i >> 1;
    const bool even = (i & 1) == 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float d[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(64 * hs + 32 * j), d);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float mine0 = d[2 * q], mine1 = d[2 * q + 1];
        const float oth0 = __shfl_xor_sync(0xffffffffu, mine0, 1);
        const float oth1 = __shfl_xor_sync(0xffffffffu, mine1, 1);
        if ((q & 1) == (even ? 0 : 1)) {
          // X_r conj(X_c) = (Re_r Re_c + Im_r Im_c) + i (Im_r Re_c - Re_r Im_c)
          const float re = even ? mine0 + oth1 : oth0 + mine1;
          const float im = even ? oth0 - mine1 : mine0 - oth1;
          stg[rho * STG_LD + 32 * hs + 16 * j + q] = make_float2(re, im);
        }
      }
    }
    tc::fence_before();
    __syncthreads();                             // staging complete
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, rr = e >> 6, q = e & 63;
      const int64_t row = r0 + rr, col = c0 + q;
      if (row < P && col < P && (!diag || q <= rr)) {
        const float2 f = stg[rr * STG_LD + q];
        float2 a = cur[u];
        a.x -= f.x;
        if (row != col) a.y -= f.y;              // the diagonal stays real
        A[row * P + col] = a;
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Factorisation of one 512-wide panel (columns p0 .. pend, all rows below) in a single
// cooperative launch, as a dataflow without grid barriers.  Blocks of 64 rows/columns are
// numbered from p0 (block g = rows p0 + 64 g ..); the panel holds blocks 0 .. ns - 1.
// Step k (k < ns) solves every row block g > k against the inverse of the diagonal block
// k, X_gk = A_gk Linv_k^H, and updates A_gc -= X_gk X_ck^H for k < c <= min(g, ns - 1).
//   * The chain CTAs 0 .. 3 take row block k + 1 through step k: once the owner of that
//     block has finished step k - 1 on it (and Linv_k is out), each solves a 16-row slab
//     and counts it on the step's ready word of the block; CTA 0 then reads the four slabs
//     and the diagonal tile, updates the tile, factors it and publishes Linv_{k+1}.  The
//     critical path per step is one slab solve, one tile update and one diagonal
//     factorisation, with no grid barrier.
//   * Every other row block g has an owner CTA, 4 + (g - 1) mod (G - 4), which runs the
//     steps k the chain does not (all k for g >= ns; k <= g - 2 for panel blocks): wait
//     for Linv_k, solve, publish the solved rows if g is a panel block (later steps' tiles
//     read them), then update its tiles on the tensor cores, waiting for each column
//     block's solved rows.  A panel block's owner reports when its step g - 2 is done.
// Owners take their blocks in ascending order within a step, and steps in order; every
// wait is on an earlier step or a smaller block, so the waits form no cycle.  Every wait is
// bounded; an expired one sets DEV_ERR_TIMEOUT and the abort word, which every wait checks.
// Sync words (zeroed before the launch): [2] the abort word, then linv[ns] (Linv_k in
// Dinv), xready[ns][ns] (step k's solved rows of block c in A: one count per chain slab
// for c = k + 1, else 1), own[ns] (step g - 2 done on panel block g).
// ---------------------------------------------------------------------------------------
constexpr int PANEL_MAX_STEPS = 8;                 // 64-column blocks per panel (NBO / 64)
constexpr int PANEL_SYNC_WORDS = 4 + PANEL_MAX_STEPS * (PANEL_MAX_STEPS + 2);
constexpr unsigned PANEL_CHAIN = 4;                // chain CTAs (16-row slabs of a block)
// the chain's tensor-core operand planes (hi, lo) sit after the factorisation's arrays
constexpr size_t CHAIN_PLANES =
    ((size_t)(3 * NB * (NB + 1) + 5 * NB) * sizeof(float2) + 1023) / 1024 * 1024;
static_assert(PANEL_SYNC_WORDS <= 128, "panel sync words");

// 16 rows r0 .. r0 + 15 of X = B L_kk^{-H} (as trsm_body); thread (row ry, columns tx + 16 b)
__device__ void trsm_slab(float2* __restrict__ A, int64_t P, int64_t k0, int kw,
                          const float2* __restrict__ Dinv, int64_t r0, unsigned char* sm,
                          const XOut& xo) {
  float2* Bt = reinterpret_cast<float2*>(sm);    // [NB (m)][17 (row)]
  float2* Lt = Bt + NB * 17;                     // [NB (m)][NB + 1 (c)]
  const int tid = threadIdx.x;
  {
    float2 bv[4], lv[16];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u, rr = e / NB, m = e % NB;
      const int64_t row = r0 + rr;
      bv[u] = (row < P && m < kw) ? __ldcg(&A[row * P + k0 + m]) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) lv[u] = __ldcg(&Dinv[tid + 256 * u]);   // e = c * NB + m
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u, rr = e / NB, m = e % NB;
      Bt[m * 17 + rr] = bv[u];
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, c = e / NB, m = e % NB;
      Lt[m * (NB + 1) + c] = lv[u];
    }
  }
  __syncthreads();
  const int ry = tid >> 4, tx = tid & 15;
  float2 acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int jb = 0; jb < 4; ++jb) {                 // Linv lower triangular (as trsm_body)
    const int mend = min(kw, 16 * jb + 16);
    for (int m = 16 * jb; m < mend; ++m) {
      const float2 br = Bt[m * 17 + ry];
#pragma unroll
      for (int q = jb; q < 4; ++q) cfmac(acc[q], br, Lt[m * (NB + 1) + tx + 16 * q]);
    }
  }
  // stage the 16 rows (over L^T, once every thread is done reading it), store coalesced
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) Lt[ry * (NB + 1) + tx + 16 * q] = acc[q];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = tid + 256 * u, r = e >> 6, c = e & 63;
    const int64_t row = r0 + r;
    if (row < P && c < kw) A[row * P + k0 + c] = Lt[r * (NB + 1) + c];
  }
  x_store_rows(xo, Lt, r0, 16, kw);
}

// CTA 0's part of a chain step: the diagonal tile of block g (rows r0 .., width kw1) less
// X X^H (X = the step's solved rows of block g, columns k0 .. k0 + kw, already in A),
// factored; L and Linv go to A and Dinv1.  The tile is read before the wait for the slabs.
// X X^H is one tensor-core product (BF16 hi/lo split of X in the swizzled operand planes at
// pl, FP32 accumulation in TMEM), folded into the tile in shared memory.  Returns false if
// a wait expired.
__device__ __noinline__ bool chain_diag(float2* __restrict__ A, int64_t P, int64_t k0, int kw, int64_t r0,
                           int kw1, float2* __restrict__ Dinv1, const unsigned* ready,
                           unsigned* abort_word, unsigned* status, unsigned char* csm,
                           uint8_t* pl, uint32_t tmem, uint32_t mbar, uint32_t* phase,
                           volatile int* tc_abort, int* issued) {
  const PotrfSmem<float2> sm(csm);
  float2* X = sm.tt;                             // [64][PLD]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  potrf_load<float2>(A, P, r0, kw1, sm.a);
  if (!cta_wait(ready, PANEL_CHAIN, abort_word, status)) return false;
  {
    float2 xv[NB * NB / 256];
    ptc_load(A, P, k0, kw, r0, xv);
    ptc_put(xv, X);                              // (PLD is the staging stride)
  }
  __syncthreads();
  ptc_pack(X, pl, pl + ptc::OP);
  tc::fence_before();
  __syncthreads();
  if (tid == 0) {
    tc::fence_after();
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 128);
    const uint64_t h = tc::smem_desc_sw128(tc::smem_u32(pl));
    const uint64_t l = tc::smem_desc_sw128(tc::smem_u32(pl + ptc::OP));
#pragma unroll
    for (int kk = 0; kk < NB / 16; ++kk) {
      const uint64_t o = (uint64_t)(kk * 32) >> 4;
      tc::mma_bf16(tmem, h + o, h + o, idesc, kk > 0 ? 1u : 0u);
      tc::mma_bf16(tmem, h + o, l + o, idesc, 1u);
      tc::mma_bf16(tmem, l + o, h + o, idesc, 1u);
    }
    tc::mma_commit(mbar);
    *issued = 1;
  }
  const bool okw = tc::warp_wait(mbar, *phase, tc_abort, lane);
  *phase ^= 1u;
  if (!__syncthreads_and(okw ? 1 : 0)) {
    if (tid == 0) {
      atomicExch(abort_word, 1u);
      flag_error(status, DEV_ERR_TIMEOUT);
    }
    return false;
  }
  tc::fence_after();
  // fold (as in herk_row_tc) straight into the tile: entry (rho, col) with col <= rho
  {
    const int qd = warp & 3, hs = warp >> 2;
    const int i = 32 * qd + lane, rho = i >> 1;
    const bool even = (i & 1) == 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float d[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(64 * hs + 32 * j), d);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float mine0 = d[2 * q], mine1 = d[2 * q + 1];
        const float oth0 = __shfl_xor_sync(0xffffffffu, mine0, 1);
        const float oth1 = __shfl_xor_sync(0xffffffffu, mine1, 1);
        const int col = 32 * hs + 16 * j + q;
        if ((q & 1) == (even ? 0 : 1) && col <= rho && rho < kw1) {
          float2& t = sm.a[rho * PLD + col];
          t.x -= even ? mine0 + oth1 : oth0 + mine1;
          if (col != rho) t.y -= even ? oth0 - mine1 : mine0 - oth1;
        }
      }
    }
  }
  tc::fence_before();
  potrf_core<float2>(status, sm);                // (begins with a barrier)
  potrf_store<float2>(A, P, r0, kw1, Dinv1, sm.a, sm.li);
  return true;
}

__global__ void __launch_bounds__(256) k_panel_coop(float2* __restrict__ A, int64_t P,
                                                    int64_t p0, int64_t pend,
                                                    float2* __restrict__ Dinv,
                                                    unsigned* sync, unsigned* status,
                                                    XOut xpanel) {
  extern __shared__ unsigned char csm_raw[];
  unsigned char* csm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(csm_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t tc_bar[2];                 // products done; drain after an abort
  __shared__ uint32_t tc_slot;
  __shared__ int tc_abort;
  const unsigned G = gridDim.x, b = blockIdx.x;
  const int ns = (int)((pend - p0 + NB - 1) / NB);
  const int NG = (int)((P - p0 + NB - 1) / NB); // row blocks from p0
  unsigned* abort_word = sync + 2;
  unsigned* linv = sync + 4;                     // [ns]
  unsigned* xready = linv + PANEL_MAX_STEPS;     // [ns][ns]
  unsigned* own = xready + PANEL_MAX_STEPS * PANEL_MAX_STEPS;   // [ns]
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&tc_bar[0]), 1);
    tc::mbar_init(tc::smem_u32(&tc_bar[1]), 1);
    tc_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(tc::smem_u32(&tc_slot)), "r"(ptc::TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tc_slot;
  uint32_t tc_phase = 0;
  int tc_issued = 0;
  auto blk_w = [&](int g) { return (int)min((int64_t)NB, P - (p0 + (int64_t)g * NB)); };
  auto xo_of = [&](int k) { XOut xo = xpanel; xo.m0 = k * NB; return xo; };
  auto dinv_of = [&](int g) { return Dinv + ((p0 + (int64_t)g * NB) / NB) * NB * NB; };

  if (b < PANEL_CHAIN) {
    // ---------------- the chain ----------------
    bool ok = true;
    if (b == 0) {
      potrf_body<float2>(A, P, p0, blk_w(0), dinv_of(0), status, csm);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicExch(&linv[0], 1u);
    }
    for (int k = 0; ok && k + 1 < ns; ++k) {
      const int g = k + 1;
      if (k >= 1 && !cta_wait(&own[g], 1u, abort_word, status)) break;
      if (b != 0 && !cta_wait(&linv[k], 1u, abort_word, status)) break;
      const int64_t k0 = p0 + (int64_t)k * NB, r0 = p0 + (int64_t)g * NB;
      trsm_slab(A, P, k0, blk_w(k), dinv_of(k), r0 + 16 * (int64_t)b, csm, xo_of(k));
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(&xready[k * PANEL_MAX_STEPS + g], 1u);
      if (b == 0) {
        ok = chain_diag(A, P, k0, blk_w(k), r0, blk_w(g), dinv_of(g),
                        &xready[k * PANEL_MAX_STEPS + g], abort_word, status, csm,
                        csm + CHAIN_PLANES, tmem, tc::smem_u32(&tc_bar[0]), &tc_phase,
                        &tc_abort, &tc_issued);
        if (!ok) break;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(&linv[g], 1u);
      }
    }
  } else if (G > PANEL_CHAIN) {
    // ---------------- row-block owners ----------------
    const int W = (int)(G - PANEL_CHAIN);
    bool ok = true;
    for (int k = 0; ok && k < ns; ++k) {
      bool waited = false;
      for (int g = 1 + (int)(b - PANEL_CHAIN); ok && g < NG; g += W) {
        if (g <= k || (g < ns && k > g - 2)) continue;   // solved, or the chain's step
        if (!waited) {
          if (!cta_wait(&linv[k], 1u, abort_word, status)) { ok = false; break; }
          waited = true;
        }
        const int64_t k0 = p0 + (int64_t)k * NB;
        const int kw = blk_w(k);
        trsm_body<float2>(A, P, k0, kw, dinv_of(k), p0 + (int64_t)g * NB, csm, xo_of(k));
        __threadfence();
        __syncthreads();
        if (g < ns && threadIdx.x == 0) atomicExch(&xready[k * PANEL_MAX_STEPS + g], 1u);
        ok = herk_row_tc(A, P, k0, kw, p0, g, k + 1, min(g, ns - 1),
                         &xready[k * PANEL_MAX_STEPS], PANEL_CHAIN, csm, tmem,
                         tc::smem_u32(&tc_bar[0]), &tc_phase, &tc_abort, &tc_issued, abort_word,
                         status);
        if (ok && g < ns && k == g - 2) {
          __threadfence();
          __syncthreads();
          if (threadIdx.x == 0) atomicExch(&own[g], 1u);
        }
      }
    }
  }
  // products still in flight after an expired wait finish before the tensor memory is
  // freed (bounded)
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && tc_abort && tc_issued) {
    volatile int dummy = 0;
    tc::mma_commit(tc::smem_u32(&tc_bar[1]));
    tc::mbar_wait(tc::smem_u32(&tc_bar[1]), 0, &dummy);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(ptc::TMEM_COLS) : "memory");
  }
}

constexpr size_t PANEL_SMEM = 1024 + CHAIN_PLANES + 2 * ptc::OP;
static_assert(PANEL_SMEM >= 1024 + ptc::SMEM, "panel shared memory holds the tensor-core tiles");

// Steps of SB = 256 rows.  After the factorisation the inverse of every 256 x 256 diagonal
// block is formed once (k_inv_sb); each block of the cooperative solve then applies it to
// the step's right-hand side redundantly (a coalesced matrix-vector product) and updates
// its share of the remaining rows; one grid barrier per step.
constexpr int SB = 256;

// Inverse of each 256 x 256 diagonal block of L, assembled from the inverses D_i of its
// four 64 x 64 diagonal blocks (left by the factorisation) by block forward substitution:
//   X_jj = D_j,   X_ij = -D_i sum_{k=j}^{i-1} L_ik X_kj   (i > j, 64 x 64 blocks),
// one CTA per (256-block, 64-column block) doing the column's 64 x 64 complex products in
// shared memory (4 x 4 register tiles): the block columns of an inverse are independent.
// Stored twice: Tb[r][c] = Linv[r][c] (backward solve) and Tf[c][r] = Linv[r][c] (forward
// solve), both [nsb][SB][SB].
template <typename C>
__device__ void tile_load(C* sm_t, const C* __restrict__ g, int64_t ld, int rows, int cols,
                          bool transpose) {
  // sm_t[m][r] (transpose) or sm_t[r][m], 64 x 65 padded; entries outside rows x cols are 0
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, m = e % NB;
    const C v = (r < rows && m < cols) ? g[(int64_t)r * ld + m] : mk<C>(0.0, 0.0);
    if (transpose) sm_t[m * (NB + 1) + r] = v;
    else sm_t[r * (NB + 1) + m] = v;
  }
}

template <typename C>
__global__ void __launch_bounds__(256) k_inv_sb(const C* __restrict__ A, int64_t P,
                                               const C* __restrict__ Dinv, C* __restrict__ Tf,
                                               C* __restrict__ Tb) {
  extern __shared__ unsigned char ism[];
  C* At = reinterpret_cast<C*>(ism);          // left operand, transposed: At[m][r]
  C* Bs = At + NB * (NB + 1);                 // right operand: Bs[m][c]
  const int sb = blockIdx.x, j = blockIdx.y;      // 256-block, and its 64-column block j
  const int64_t k0 = (int64_t)sb * SB;
  const int kw = (int)min((int64_t)SB, P - k0);
  const int nblk = (kw + NB - 1) / NB;
  C* tb = Tb + (int64_t)sb * SB * SB;
  C* tf = Tf + (int64_t)sb * SB * SB;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // column block j: the diagonal block and zeros elsewhere
  for (int e = tid; e < SB * NB; e += 256) {
    const int r = e / NB, c = NB * j + e % NB, i = r / NB;
    tb[(int64_t)r * SB + c] =
        (i == j && i < nblk) ? Dinv[((int64_t)(k0 / NB) + i) * NB * NB + (r % NB) * NB + (c % NB)]
                             : mk<C>(0.0, 0.0);
  }
  __syncthreads();
  auto rows_of = [&](int i) { return min(NB, kw - NB * i); };
  if (j < nblk) {
    for (int i = j + 1; i < nblk; ++i) {
      C acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk<C>(0.0, 0.0);
      // T = sum_k L_ik X_kj
      for (int k = j; k < i; ++k) {
        tile_load(At, A + (k0 + NB * i) * P + k0 + NB * k, P, rows_of(i), rows_of(k), true);
        tile_load(Bs, tb + (int64_t)(NB * k) * SB + NB * j, SB, rows_of(k), rows_of(j), false);
        __syncthreads();
        for (int m = 0; m < NB; ++m) {
          C ar[4], bc[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) ar[a] = At[m * (NB + 1) + ty + 16 * a];
#pragma unroll
          for (int b = 0; b < 4; ++b) bc[b] = Bs[m * (NB + 1) + tx + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) cfma(acc[a][b], ar[a], bc[b]);
        }
        __syncthreads();
      }
      // X_ij = -D_i T
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) Bs[(ty + 16 * a) * (NB + 1) + tx + 16 * b] = acc[a][b];
      tile_load(At, Dinv + ((int64_t)(k0 / NB) + i) * NB * NB, NB, NB, NB, true);
      __syncthreads();
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk<C>(0.0, 0.0);
      for (int m = 0; m < NB; ++m) {
        C ar[4], bc[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) ar[a] = At[m * (NB + 1) + ty + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bc[b] = Bs[m * (NB + 1) + tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) cfma(acc[a][b], ar[a], bc[b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int r = ty + 16 * a, c = tx + 16 * b;
          C v = acc[a][b];
          v.x = -v.x;
          v.y = -v.y;
          if (r < rows_of(i) && c < rows_of(j)) tb[(int64_t)(NB * i + r) * SB + NB * j + c] = v;
        }
      __syncthreads();
    }
  }
  for (int e = tid; e < SB * NB; e += 256) {
    const int r = e % SB, c = NB * j + e / SB;
    tf[(int64_t)c * SB + r] = tb[(int64_t)r * SB + c];
  }
}

// ---------------------------------------------------------------------------------------
// Triangular solves as a dataflow over 32-row slices, one cooperative launch each.  The
// right-hand side is cut into slices (j, s) = rows 256 j + 32 s .. + 31 of 256-row block j;
// each slice has a fixed owner CTA (slice index mod grid), which applies all of the
// slice's block updates in order.  Forward step k (L y = b):
//   * the owners of block k's eight slices read the block's final right-hand side, each
//     computes its 32 entries of y_k = Linv_kk b_k (Linv_kk from the precomputed 256 x 256
//     inverses) and stores them;
//   * the owner of every slice of a later block subtracts L[rows][block k] y_k from its
//     rows; the last of these updates (block k + 1) goes to the final buffer.
// The backward solve (L^H x = y) runs the same scheme from the last block to the first with
// x_k = Linv_kk^H c_k and the rows above.  The data are their own flags: the solution and
// the final buffer are filled with an all-ones bit pattern (a NaN that arithmetic does not
// produce) before the launch, every entry is written once, and a reader polls the entries
// it needs until no component holds the pattern.  There is no counter, flag or fence on
// the critical path, which is the eight-CTA product and two polled reads per block.  Every
// wait is bounded (iteration and clock limits); an expired wait sets DEV_ERR_TIMEOUT and
// the abort word, which every other wait also checks.  Right-hand sides go through L2
// only (ld/st.global.cg, volatile polls).
// ---------------------------------------------------------------------------------------
constexpr int TS = 32;                          // slice rows
constexpr int SPB = SB / TS;                    // slices per 256-row block

// One component word of a right-hand-side entry; all ones marks "not written yet".
template <typename C> struct WordOf;
template <> struct WordOf<float2> { typedef unsigned T; };
template <> struct WordOf<double2> { typedef unsigned long long T; };

// Wait (bounded) until both components of *p are written, and return the entry.
template <typename C>
__device__ __forceinline__ bool poll_entry(const C* p, C* out, unsigned* abort_word,
                                           unsigned* status) {
  typedef typename WordOf<C>::T W;
  const W NONE = ~(W)0;
  volatile const W* w = reinterpret_cast<volatile const W*>(p);
  volatile unsigned* vab = abort_word;
  const long long t0 = clock64();
  unsigned it = 0;
  for (;;) {
    const W x = w[0], y = w[1];
    if (x != NONE && y != NONE) {
      W* o = reinterpret_cast<W*>(out);
      o[0] = x;
      o[1] = y;
      return true;
    }
    if (*vab) return false;
    if ((++it & 255u) == 0 && clock64() - t0 > 2000000000ll) {
      atomicExch(abort_word, 1u);
      flag_error(status, DEV_ERR_TIMEOUT);
      return false;
    }
  }
}

// dst[t] = src[t] for t < n, waiting for each entry; CTA-wide verdict
template <typename C>
__device__ __forceinline__ bool cta_poll_block(const C* src, C* dst, int n, unsigned* abort_word,
                                               unsigned* status) {
  bool ok = true;
  const int t = threadIdx.x;
  if (t < n) ok = poll_entry<C>(&src[t], &dst[t], abort_word, status);
  else if (t < SB) dst[t] = mk<C>(0.0, 0.0);
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// this CTA's 32 entries [32 s, 32 s + 32) of y = T^(op) v for the 256 x 256 block T
// (T[m][t]; CONJ: conj(T)); v in shared memory; result to out (L2).  The block's entries
// are loaded first (slice_load, before the waits: T is read-only during the solve).
template <typename C>
__device__ __forceinline__ void slice_load(const C* __restrict__ T, int s, C (&w)[32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = TS * s + lane;
#pragma unroll
  for (int j = 0; j < 32; ++j) w[j] = __ldg(&T[(int64_t)(32 * warp + j) * SB + t]);
}

template <typename C, bool CONJ>
__device__ __forceinline__ void slice_matvec(const C (&w)[32], const C* vv, int s, int kw,
                                             C* out, C* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = TS * s + lane;
  C acc = mk<C>(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (CONJ) cfmac(acc, vv[32 * warp + j], w[j]);
    else cfma(acc, w[j], vv[32 * warp + j]);
  }
  red[warp * 32 + lane] = acc;
  __syncthreads();
  if (warp == 0) {
    C tot = red[lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) { tot.x += red[q * 32 + lane].x; tot.y += red[q * 32 + lane].y; }
    if (t < kw) __stcg(&out[t], tot);
  }
  __syncthreads();
}

// sync: [0] abort word.  y (and fin) hold the all-ones pattern at launch; fin receives the
// final right-hand side of every block after the first.
template <typename C>
__global__ void __launch_bounds__(256) k_fwd_coop(const C* __restrict__ A,
                                                  const C* __restrict__ Tf, int64_t P,
                                                  C* __restrict__ b, C* __restrict__ y,
                                                  C* __restrict__ fin, unsigned* sync,
                                                  unsigned* status) {
  __shared__ C vv[SB];
  __shared__ C red[SB];
  __shared__ C yk[SB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsb = (int)((P + SB - 1) / SB);
  const int G = gridDim.x, me = blockIdx.x;
  unsigned* abort_word = sync;
  const int nslices = nsb * SPB;
  for (int k = 0; k < nsb; ++k) {
    const int64_t k0 = (int64_t)k * SB;
    const int kw = (int)min((int64_t)SB, P - k0);
    // 1. owners of block k's slices: y_k
    for (int s = 0; s < SPB; ++s) {
      const int q = k * SPB + s;
      if (q % G != me) continue;
      C w[32];
      slice_load<C>(Tf + (int64_t)k * SB * SB, s, w);
      if (k == 0) {
        vv[tid] = (tid < kw) ? __ldcg(&b[tid]) : mk<C>(0.0, 0.0);
        __syncthreads();
      } else if (!cta_poll_block<C>(fin + k0, vv, kw, abort_word, status)) {
        return;
      }
      slice_matvec<C, false>(w, vv, s, kw, y + k0, red);
    }
    // 2. owners of later slices: b_rows -= L[rows][block k] y_k
    bool have_y = false;
    for (int q = me; q < nslices; q += G) {
      const int j = q / SPB, s = q % SPB;
      if (j <= k) continue;
      const int64_t r0 = (int64_t)j * SB + (int64_t)s * TS;
      if (r0 >= P) continue;
      // four rows per warp, lanes over the 256 columns (8 each); L and the slice's own
      // rows of b (written only by this CTA) are loaded before the wait for y_k
      C v[4][8];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int m = lane + 32 * i;
          const int64_t row = r0 + warp * 4 + rr;
          v[rr][i] = (row < P && m < kw) ? A[row * P + k0 + m] : mk<C>(0.0, 0.0);
        }
      C cur = mk<C>(0.0, 0.0);
      if (lane < 4 && r0 + warp * 4 + lane < P) cur = __ldcg(&b[r0 + warp * 4 + lane]);
      if (!have_y) {
        if (!cta_poll_block<C>(y + k0, yk, kw, abort_word, status)) return;
        have_y = true;
      }
      C* dst = (j == k + 1) ? fin : b;             // block k+1's last update is final
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        C sacc = mk<C>(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < 8; ++i) cfma(sacc, v[rr][i], yk[lane + 32 * i]);
        for (int o = 16; o > 0; o >>= 1) {
          sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
          sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
        }
        const int64_t row = r0 + warp * 4 + rr;
        if (lane == rr && row < P) {
          C t = cur;
          t.x -= sacc.x;
          t.y -= sacc.y;
          __stcg(&dst[row], t);
        }
      }
    }
    if (have_y) __syncthreads();                   // yk is rewritten at the next step
  }
}

// sync: [0] abort word.  x (and fin) hold the all-ones pattern at launch; fin receives the
// final right-hand side of every block before the last.
template <typename C>
__global__ void __launch_bounds__(256) k_bwd_coop(const C* __restrict__ A,
                                                  const C* __restrict__ Tb, int64_t P,
                                                  C* __restrict__ c, C* __restrict__ x,
                                                  C* __restrict__ fin, unsigned* sync,
                                                  unsigned* status) {
  __shared__ C vv[SB];
  __shared__ C red[SB];
  __shared__ C xk[SB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsb = (int)((P + SB - 1) / SB);
  const int G = gridDim.x, me = blockIdx.x;
  unsigned* abort_word = sync;
  const int nslices = nsb * SPB;
  for (int k = nsb - 1; k >= 0; --k) {
    const int64_t k0 = (int64_t)k * SB;
    const int kw = (int)min((int64_t)SB, P - k0);
    for (int s = 0; s < SPB; ++s) {
      const int q = k * SPB + s;
      if (q % G != me) continue;
      C w[32];
      slice_load<C>(Tb + (int64_t)k * SB * SB, s, w);
      if (k == nsb - 1) {
        vv[tid] = (tid < kw) ? __ldcg(&c[k0 + tid]) : mk<C>(0.0, 0.0);
        __syncthreads();
      } else if (!cta_poll_block<C>(fin + k0, vv, kw, abort_word, status)) {
        return;
      }
      slice_matvec<C, true>(w, vv, s, kw, x + k0, red);
    }
    // owners of earlier slices: c_rows -= L[block k][rows]^H x_k; lanes over the 32 rows,
    // warp w over the columns [32 w, 32 w + 32) of block k, shared-memory reduction
    bool have_x = false;
    for (int q = me; q < nslices; q += G) {
      const int j = q / SPB, s = q % SPB;
      if (j >= k) continue;
      const int64_t r0 = (int64_t)j * SB + (int64_t)s * TS;
      const int64_t r = r0 + lane;                 // r < k0 <= P
      C v[32];                                     // loaded before the wait for x_k
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const int m = warp * 32 + jj;
        v[jj] = (m < kw) ? A[(k0 + m) * P + r] : mk<C>(0.0, 0.0);
      }
      const C cur = (warp == 0) ? __ldcg(&c[r]) : mk<C>(0.0, 0.0);
      if (!have_x) {
        if (!cta_poll_block<C>(x + k0, xk, kw, abort_word, status)) return;
        have_x = true;
      }
      C sacc = mk<C>(0.0, 0.0);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) cfmac(sacc, xk[warp * 32 + jj], v[jj]);
      red[warp * 32 + lane] = sacc;
      __syncthreads();
      if (warp == 0) {
        C tot = red[lane];
#pragma unroll
        for (int w = 1; w < 8; ++w) { tot.x += red[w * 32 + lane].x; tot.y += red[w * 32 + lane].y; }
        C t = cur;
        t.x -= tot.x;
        t.y -= tot.y;
        __stcg((j == k - 1) ? &fin[r] : &c[r], t);  // block k-1's last update is final
      }
      __syncthreads();
    }
    if (have_x) __syncthreads();
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

// b = D a (D the equilibration scales, or 1 when dsc is null)
__global__ void k_to_f32(const double2* __restrict__ a, float2* __restrict__ b, int64_t P,
                         const float* __restrict__ dsc) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const double d = dsc ? (double)dsc[k] : 1.0;
    b[k] = make_float2((float)(a[k].x * d), (float)(a[k].y * d));
  }
}

// x += D c
__global__ void k_add_f32(double2* __restrict__ x, const float2* __restrict__ c, int64_t P,
                          const float* __restrict__ dsc) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const double d = dsc ? (double)dsc[k] : 1.0;
    x[k].x += (double)c[k].x * d;
    x[k].y += (double)c[k].y * d;
  }
}

// Jacobi equilibration of the factor's input: d_k = 1 / sqrt(A_kk), A_rc <- d_r A_rc d_c on
// the lower triangle (unit diagonal).  The FP32 factorisation of S~ with its diagonal
// spread over orders of magnitude (Var s_i ~ 1 against |t_j|^2 << 1) keeps positive pivots
// and contracts the refinement faster on the scaled matrix; corrections are mapped back
// with D (S~ c = r  <=>  (D S~ D)(D^-1 c) = D r).
__global__ void k_eq_scales(const float2* __restrict__ A, int64_t P, float* __restrict__ dsc) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    const float d = A[k * P + k].x;
    dsc[k] = (d > 0.f && isfinite(d)) ? rsqrtf(d) : 1.f;
  }
}

// one block per row r: the lower part c <= r, coalesced along the row
__global__ void k_equilibrate(float2* __restrict__ A, int64_t P, const float* __restrict__ dsc) {
  const int64_t r = blockIdx.x;
  const float dr = dsc[r];
  float2* row = A + r * P;
  for (int64_t c = threadIdx.x; c <= r; c += blockDim.x) {
    const float s = dr * dsc[c];
    float2 v = row[c];
    v.x *= s;
    v.y *= s;
    row[c] = v;
  }
}

__global__ void k_update(double2* __restrict__ p, const double2* __restrict__ x, int64_t P, double dt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    p[k].x -= dt * x[k].x;
    p[k].y -= dt * x[k].y;
  }
}

// ---------------------------------------------------------------------------------------
// Residuals of the mixed solvers in compensated FP32 arithmetic.  S and x are held as
// FP32 hi/lo pairs (S = S_hi + S_lo to ~2^-48); each row's sum of S_hi x_hi products is
// accumulated error-free (Dekker's product by fma, Knuth's two-sum) into a (sum,
// correction) pair, the hi.lo and lo.hi terms (2^-24 smaller) into the correction.  This
// keeps the refinement at FP64-level accuracy on the FP32 pipe (FP64 throughput on this
// part is ~1/60 of FP32).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float p) {
  const float t = s + p;
  const float bb = t - s;
  c += (s - (t - bb)) + (p - bb);
  s = t;
}

__global__ void k_split_x(const double2* __restrict__ x, float4* __restrict__ x2, int64_t P) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[k];
    const float hr = (float)v.x, hi = (float)v.y;
    x2[k] = make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
  }
}

// S (FP64) -> S2 (hi/lo pairs, every entry) and A32 (lower triangle, shifted diagonal)
__global__ void k_split_shift(const double2* __restrict__ S, float4* __restrict__ S2,
                              float2* __restrict__ A, int64_t P, double nu, int mode) {
  const int64_t total = P * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = S[e];
    const float hr = (float)v.x, hi = (float)v.y;
    S2[e] = make_float4(hr, hi, (float)(v.x - (double)hr), (float)(v.y - (double)hi));
    const int64_t r = e / P, c = e - r * P;
    if (c <= r) {
      const float d = (r == c) ? (float)(mode == 0 ? v.x * (1.0 + nu) : v.x + nu) : hr;
      A[e] = make_float2(d, hi);
    }
  }
}

// A32 (lower, shifted) again from S2, for a refactorisation
__global__ void k_s2_to_a32(const float4* __restrict__ S2, float2* __restrict__ A, int64_t P,
                            double nu, int mode) {
  const int64_t total = P * P;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / P, c = e - r * P;
    if (c > r) continue;
    const float4 v = S2[e];
    float d = v.x;
    if (r == c) {
      const double s = (double)v.x + (double)v.z;
      d = (float)(mode == 0 ? s * (1.0 + nu) : s + nu);
    }
    A[e] = make_float2(d, v.y);
  }
}

// r = F - (S + shift) x, one block per row; acc[0] += ||r||^2
__global__ void __launch_bounds__(256) k_resid_df(const float4* __restrict__ S2,
                                                  const float4* __restrict__ x2,
                                                  const double2* __restrict__ x,
                                                  const double2* __restrict__ F, int64_t P,
                                                  double nu, int mode, double2* __restrict__ r,
                                                  double* acc) {
  __shared__ double red[2][8];
  const int64_t row = blockIdx.x;
  const float4* srow = S2 + row * P;
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
#pragma unroll 4
  for (int64_t c = threadIdx.x; c < P; c += blockDim.x) {
    const float4 a = __ldcs(&srow[c]);   // hi.re, hi.im, lo.re, lo.im (streamed once)
    const float4 v = x2[c];
    const float p1 = a.x * v.x, e1 = fmaf(a.x, v.x, -p1);
    const float p2 = -(a.y * v.y), e2 = fmaf(-a.y, v.y, -p2);
    const float p3 = a.x * v.y, e3 = fmaf(a.x, v.y, -p3);
    const float p4 = a.y * v.x, e4 = fmaf(a.y, v.x, -p4);
    float tr = e1 + e2;
    tr = fmaf(a.x, v.z, tr);
    tr = fmaf(-a.y, v.w, tr);
    tr = fmaf(a.z, v.x, tr);
    tr = fmaf(-a.w, v.y, tr);
    float ti = e3 + e4;
    ti = fmaf(a.x, v.w, ti);
    ti = fmaf(a.y, v.z, ti);
    ti = fmaf(a.z, v.y, ti);
    ti = fmaf(a.w, v.x, ti);
    two_sum_acc(sr, cr, p1);
    two_sum_acc(sr, cr, p2);
    cr += tr;
    two_sum_acc(si, ci, p3);
    two_sum_acc(si, ci, p4);
    ci += ti;
  }
  double dr = (double)sr + (double)cr, di = (double)si + (double)ci;
  dr = warp_sum_d(dr);
  di = warp_sum_d(di);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[0][w] = dr; red[1][w] = di; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0, ti = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { tr += red[0][k]; ti += red[1][k]; }
    const float4 d = srow[row];
    const double skk = (double)d.x + (double)d.z;
    const double2 v = x[row];
    const double extra = (mode == 0) ? nu * skk : nu;   // shift acts on the diagonal only
    tr += extra * v.x;
    ti += extra * v.y;
    const double2 f = F[row];
    const double2 res = make_double2(f.x - tr, f.y - ti);
    r[row] = res;
    atomicAdd(acc, res.x * res.x + res.y * res.y);
  }
}

// Failure-path self-test: the cooperative kernels' bounded flag wait on a word that nothing
// sets (word[0] = 0, word[1] = the abort word) must give up, set DEV_ERR_TIMEOUT and return.
__global__ void k_selftest_flag_wait(unsigned* word, unsigned* status) {
  if (threadIdx.x == 0) wait_at_least(word, 1u, word + 1, status);
}

cudaError_t launch_selftest_flag_wait(unsigned* word2, unsigned* status, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(word2, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_selftest_flag_wait<<<1, 32, 0, st>>>(word2, status);
  return cudaGetLastError();
}

// ... and the triangular solves' bounded poll on an entry that nothing writes (word4[0..1]
// hold the all-ones pattern, word4[2] is the abort word).
__global__ void k_selftest_poll_wait(unsigned* word4, unsigned* status) {
  if (threadIdx.x == 0) {
    float2 v;
    poll_entry<float2>(reinterpret_cast<const float2*>(word4), &v, word4 + 2, status);
  }
}

cudaError_t launch_selftest_poll_wait(unsigned* word4, unsigned* status, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(word4, 0xff, 2 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(word4 + 2, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  k_selftest_poll_wait<<<1, 32, 0, st>>>(word4, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
template <typename C>
static constexpr size_t potrf_smem() { return (size_t)(3 * NB * (NB + 1) + 5 * NB) * sizeof(C); }

template <typename C>
static cudaError_t set_smem_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  const int s2 = 2 * NB * (NB + 1) * (int)sizeof(C);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_potrf_diag<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, potrf_smem<C>())) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_trsm_inv<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_inv_sb<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2)) != cudaSuccess) return e;
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
    k_potrf_diag<C><<<1, POTRF_THREADS, potrf_smem<C>(), st>>>(A, P, k0, kw, Dinv + kb * NB * NB, status);
    ++*launches;
    const int64_t rest = P - k0 - kw;
    if (rest > 0) {
      k_trsm_inv<C><<<(unsigned)((rest + NB - 1) / NB), 256, s2, st>>>(A, P, k0, kw, Dinv + kb * NB * NB);
      const int64_t nt = (rest + NB - 1) / NB;
      k_herk<C><<<(unsigned)(nt * (nt + 1) / 2), 256, s2, st>>>(A, P, k0, kw, P);
      *launches += 2;
    }
    VMC_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

// Two-level factorisation: 512-wide panels factored by the cooperative panel kernel (64-wide
// diagonal blocks, updates restricted to the panel's columns), then the whole trailing
// matrix receives the panel's Schur complement on the tensor cores (BF16 split, K = 512).
static constexpr int NBO = 512;
static_assert(NBO / NB <= PANEL_MAX_STEPS, "panel step counters");

static cudaError_t factor_tc(float2* A, float2* Dinv, int64_t P, SolveWork& w, unsigned* status,
                             cudaStream_t st, int64_t* launches) {
  VMC_TRY(set_smem_attrs<float2>());               // k_inv_sb and the refactorisation fallback
  static int grid = 0;
  if (grid == 0) {
    VMC_TRY(cudaFuncSetAttribute(k_panel_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PANEL_SMEM));
    int dev = 0, sms = 0, per_sm = 0;
    VMC_TRY(cudaGetDevice(&dev));
    VMC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VMC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel_coop, 256, PANEL_SMEM));
    // one CTA per SM; the chain needs at least one row-block owner beside it
    if (per_sm < 1 || sms <= (int)PANEL_CHAIN) return cudaErrorCooperativeLaunchTooLarge;
    grid = sms;
  }
  unsigned* sync = w.bar;
  for (int64_t p0 = 0; p0 < P; p0 += NBO) {
    const int64_t pend = std::min<int64_t>(P, p0 + NBO);
    // the rows below the panel go, as they are solved, into the BF16 hi/lo operand planes of
    // the panel's Schur update (rows_pad rows; the padding rows are zeroed here)
    const int64_t n = P - pend;
    const int K = (int)(pend - p0);
    const int64_t rows_pad = (2 * n + 127) / 128 * 128;
    XOut xo{nullptr, nullptr, pend, n, K, 0};
    if (n > 0) {
      if (rows_pad * NBO > w.x_elems || K != NBO) return cudaErrorInvalidValue;
      const size_t pad = (size_t)(rows_pad - 2 * n) * K * sizeof(__nv_bfloat16);
      if (pad) {
        VMC_TRY(cudaMemsetAsync(w.Xhi + 2 * n * K, 0, pad, st));
        VMC_TRY(cudaMemsetAsync(w.Xlo + 2 * n * K, 0, pad, st));
      }
      xo.hi = w.Xhi;
      xo.lo = w.Xlo;
    }
    VMC_TRY(cudaMemsetAsync(sync, 0, PANEL_SYNC_WORDS * sizeof(unsigned), st));
    void* args[] = {(void*)&A,    (void*)&P,      (void*)&p0, (void*)&pend, (void*)&Dinv,
                    (void*)&sync, (void*)&status, (void*)&xo};
    VMC_TRY(cudaLaunchCooperativeKernel((const void*)k_panel_coop, dim3(grid), dim3(256), args,
                                        PANEL_SMEM, st));
    ++*launches;
    if (n > 0) {
      VMC_TRY(launch_herk_tc(w.Xhi, w.Xlo, rows_pad, K, n, A, P, pend, NBO, 3, status, st));
      ++*launches;
    }
  }
  return cudaSuccess;
}

// b is overwritten (workspace); the solution lands in x.  One cooperative launch per
// substitution (all blocks resident: the grid is sized from the occupancy query).
template <typename C> static C* inv_fwd(SolveWork& w);
template <> float2* inv_fwd<float2>(SolveWork& w) { return w.T32f; }
template <> double2* inv_fwd<double2>(SolveWork& w) { return w.T64f; }
template <typename C> static C* inv_bwd(SolveWork& w);
template <> float2* inv_bwd<float2>(SolveWork& w) { return w.T32b; }
template <> double2* inv_bwd<double2>(SolveWork& w) { return w.T64b; }

template <typename C> static const C* dinv_of(SolveWork& w);
template <> const float2* dinv_of<float2>(SolveWork& w) { return w.D32; }
template <> const double2* dinv_of<double2>(SolveWork& w) { return w.D64; }

// inverses of the 256-wide diagonal blocks of the factor (once per factorisation)
template <typename C>
static cudaError_t invert_blocks(const C* A, int64_t P, SolveWork& w, cudaStream_t st,
                                 int64_t* launches) {
  const int64_t nsb = (P + SB - 1) / SB;
  const C* Dinv = dinv_of<C>(w);
  k_inv_sb<C><<<dim3((unsigned)nsb, SB / NB), 256, 2 * NB * (NB + 1) * sizeof(C), st>>>(A, P, Dinv, inv_fwd<C>(w),
                                                                           inv_bwd<C>(w));
  ++*launches;
  return cudaGetLastError();
}

template <typename C>
static cudaError_t chol_solve(const C* A, const C* Dinv_unused, int64_t P, C* b, C* y, C* x,
                              SolveWork& w, unsigned* status, cudaStream_t st, int64_t* launches) {
  (void)Dinv_unused;
  const C* Dinv = inv_fwd<C>(w);   // forward kernel reads the transposed inverses
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    VMC_TRY(cudaGetDevice(&dev));
    VMC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int pf = 0, pb = 0;
    VMC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, k_fwd_coop<C>, 256, 0));
    VMC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pb, k_bwd_coop<C>, 256, 0));
    per_sm = std::min(std::min(pf, pb), 1);
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    grid = sms * per_sm;
  }
  // w.bar[0]: abort word; outputs and the final buffer start as the all-ones pattern
  unsigned* sync = w.bar;
  C* fin = reinterpret_cast<C*>(w.fin);
  const size_t vbytes = (size_t)P * sizeof(C);
  VMC_TRY(cudaMemsetAsync(sync, 0, sizeof(unsigned), st));
  VMC_TRY(cudaMemsetAsync(y, 0xff, vbytes, st));
  VMC_TRY(cudaMemsetAsync(fin, 0xff, vbytes, st));
  {
    void* args[] = {(void*)&A, (void*)&Dinv, (void*)&P, (void*)&b, (void*)&y, (void*)&fin,
                    (void*)&sync, (void*)&status};
    VMC_TRY(cudaLaunchCooperativeKernel((const void*)k_fwd_coop<C>, dim3(grid), dim3(256), args, 0, st));
  }
  VMC_TRY(cudaMemsetAsync(sync, 0, sizeof(unsigned), st));
  VMC_TRY(cudaMemsetAsync(x, 0xff, vbytes, st));
  VMC_TRY(cudaMemsetAsync(fin, 0xff, vbytes, st));
  {
    const C* Dinvb = inv_bwd<C>(w);
    void* args[] = {(void*)&A, (void*)&Dinvb, (void*)&P, (void*)&y, (void*)&x, (void*)&fin,
                    (void*)&sync, (void*)&status};
    VMC_TRY(cudaLaunchCooperativeKernel((const void*)k_bwd_coop<C>, dim3(grid), dim3(256), args, 0, st));
  }
  *launches += 2;
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
  VMC_TRY(invert_blocks<double2>(w.A64, P, w, st, launches));
  VMC_TRY(cudaMemcpyAsync(w.c, F, P * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  return chol_solve<double2>(w.A64, w.D64, P, w.c, w.r, x, w, status, st, launches);
}

cudaError_t split_shift(const double2* S, double nu, int mode, SolveWork& w, cudaStream_t st) {
  k_split_shift<<<grid_for(w.P * w.P, 256), 256, 0, st>>>(S, w.S2, w.A32, w.P, nu, mode);
  return cudaGetLastError();
}

static cudaError_t residual_df(const double2* F, const double2* x, double nu, int mode,
                               SolveWork& w, cudaStream_t st, double* relres) {
  const int64_t P = w.P;
  VMC_TRY(cudaMemsetAsync(w.scal, 0, 2 * sizeof(double), st));
  k_split_x<<<grid_for(P, 256, 1024), 256, 0, st>>>(x, w.x2, P);
  k_resid_df<<<(unsigned)P, 256, 0, st>>>(w.S2, w.x2, x, F, P, nu, mode, w.r, w.scal);
  k_norm2<<<grid_for(P, 256, 1024), 256, 0, st>>>(F, P, w.scal + 1);
  VMC_TRY(cudaGetLastError());
  double h[2];
  VMC_TRY(cudaMemcpyAsync(h, w.scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  VMC_TRY(cudaStreamSynchronize(st));
  *relres = (h[1] > 0) ? sqrt(h[0] / h[1]) : 0.0;
  return cudaSuccess;
}

cudaError_t solve_cholesky_mixed(const double2* F, double2* x, double nu, int mode, double tol,
                                 int maxit, bool tc, SolveWork& w, unsigned* status,
                                 cudaStream_t st, int64_t* launches, int* iters,
                                 double* relres) {
  const int64_t P = w.P;
  k_eq_scales<<<grid_for(P, 256, 1024), 256, 0, st>>>(w.A32, P, w.dsc);
  k_equilibrate<<<(unsigned)P, 256, 0, st>>>(w.A32, P, w.dsc);
  *launches += 2;
  if (tc && P > NBO) VMC_TRY(factor_tc(w.A32, w.D32, P, w, status, st, launches));
  else VMC_TRY(factor<float2>(w.A32, w.D32, P, status, st, launches));
  VMC_TRY(invert_blocks<float2>(w.A32, P, w, st, launches));
  VMC_TRY(cudaMemsetAsync(x, 0, P * sizeof(double2), st));
  VMC_TRY(cudaMemcpyAsync(w.r, F, P * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  double rel = 1.0, prev = 1.0;
  bool tc_factor = tc && P > NBO;
  int it = 0;
  for (; it < std::max(1, maxit); ++it) {
    k_to_f32<<<grid_for(P, 256, 1024), 256, 0, st>>>(w.r, w.r32, P, w.dsc);
    VMC_TRY(chol_solve<float2>(w.A32, w.D32, P, w.r32, w.y32, w.c32, w, status, st, launches));
    k_add_f32<<<grid_for(P, 256, 1024), 256, 0, st>>>(x, w.c32, P, w.dsc);
    *launches += 2;
    VMC_TRY(residual_df(F, x, nu, mode, w, st, &rel));
    *launches += 3;
    if (!(rel == rel)) break;      // NaN
    if (rel <= tol) { ++it; break; }
    // The BF16-split factor contracts the error by ~cond(S~) * 2^-16 per iteration; if that
    // is too slow, refactor in FP32 and keep refining from the current x.
    if (tc_factor && it >= 1 && rel > 0.25 * prev) {
      k_s2_to_a32<<<grid_for(P * P, 256), 256, 0, st>>>(w.S2, w.A32, P, nu, mode);
      k_equilibrate<<<(unsigned)P, 256, 0, st>>>(w.A32, P, w.dsc);
      *launches += 2;
      VMC_TRY(factor<float2>(w.A32, w.D32, P, status, st, launches));
      VMC_TRY(invert_blocks<float2>(w.A32, P, w, st, launches));
      tc_factor = false;
    }
    prev = rel;
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;      // the caller compares it with tol
  return cudaSuccess;
}

// ---------------------------------------------------------------------------------------
// Conjugate gradients on an exactly applied operator A (a callback), preconditioned by the
// FP32 Cholesky factor of an approximation of A held in w.A32 (lower triangle, shift
// included).  With the factor of the BF16-split S this solves the system of the samples'
// own S to the accuracy of the operator, whatever the split's rounding, since the factor
// only preconditions.  Dot products: fixed-order FP64 block partials summed on the host.
// ---------------------------------------------------------------------------------------
constexpr int PCG_DOT_BLOCKS = 128;

// part[b] = Re sum a^H b, part[nb + b] = sum |a|^2 over this block's share
__global__ void k_pcg_dots(const double2* __restrict__ a, const double2* __restrict__ b, int64_t P,
                           double* part) {
  __shared__ double s1[256], s2[256];
  double d = 0.0, n2 = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = a[k], v = b[k];
    d = fma(u.x, v.x, fma(u.y, v.y, d));
    n2 = fma(u.x, u.x, fma(u.y, u.y, n2));
  }
  s1[threadIdx.x] = d;
  s2[threadIdx.x] = n2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1[0];
    part[gridDim.x + blockIdx.x] = s2[0];
  }
}

// x += alpha p, r -= alpha q
__global__ void k_pcg_update(double2* x, double2* r, const double2* p, const double2* q,
                             double alpha, int64_t P) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    x[k].x = fma(alpha, p[k].x, x[k].x);
    x[k].y = fma(alpha, p[k].y, x[k].y);
    r[k].x = fma(-alpha, q[k].x, r[k].x);
    r[k].y = fma(-alpha, q[k].y, r[k].y);
  }
}

// p = z + beta p
__global__ void k_pcg_dir(double2* p, const double2* z, double beta, int64_t P) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    p[k] = make_double2(fma(beta, p[k].x, z[k].x), fma(beta, p[k].y, z[k].y));
  }
}

// z = D c (the equilibrated factor's correction mapped back)
__global__ void k_set_f32(double2* __restrict__ z, const float2* __restrict__ c, int64_t P,
                          const float* __restrict__ dsc) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double d = dsc ? (double)dsc[k] : 1.0;
    z[k] = make_double2((double)c[k].x * d, (double)c[k].y * d);
  }
}

// r = F - q
__global__ void k_sub(const double2* F, const double2* q, double2* r, int64_t P) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P;
       k += (int64_t)gridDim.x * blockDim.x)
    r[k] = make_double2(F[k].x - q[k].x, F[k].y - q[k].y);
}

static cudaError_t pcg_dots(const double2* a, const double2* b, int64_t P, double* part,
                            cudaStream_t st, double* dot, double* n2) {
  k_pcg_dots<<<PCG_DOT_BLOCKS, 256, 0, st>>>(a, b, P, part);
  VMC_TRY(cudaGetLastError());
  double h[2 * PCG_DOT_BLOCKS];
  VMC_TRY(cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, st));
  VMC_TRY(cudaStreamSynchronize(st));
  double d = 0.0, n = 0.0;
  for (int b2 = 0; b2 < PCG_DOT_BLOCKS; ++b2) {
    d += h[b2];
    n += h[PCG_DOT_BLOCKS + b2];
  }
  *dot = d;
  *n2 = n;
  return cudaSuccess;
}

cudaError_t solve_pcg_factor(const double2* F, double2* x, double tol, int maxit, bool tc,
                             const PcgOperator& apply, double2* r, double2* z, double2* p,
                             double2* q, SolveWork& w, unsigned* status, cudaStream_t st,
                             int64_t* launches, int* iters, double* relres, double* relres_rec) {
  const int64_t P = w.P;
  k_eq_scales<<<grid_for(P, 256, 1024), 256, 0, st>>>(w.A32, P, w.dsc);
  k_equilibrate<<<(unsigned)P, 256, 0, st>>>(w.A32, P, w.dsc);
  *launches += 2;
  if (tc && P > NBO) VMC_TRY(factor_tc(w.A32, w.D32, P, w, status, st, launches));
  else VMC_TRY(factor<float2>(w.A32, w.D32, P, status, st, launches));
  VMC_TRY(invert_blocks<float2>(w.A32, P, w, st, launches));
  const unsigned g = grid_for(P, 256, 1024);
  auto precondition = [&](const double2* rin, double2* zout) -> cudaError_t {
    k_to_f32<<<g, 256, 0, st>>>(rin, w.r32, P, w.dsc);
    VMC_TRY(chol_solve<float2>(w.A32, w.D32, P, w.r32, w.y32, w.c32, w, status, st, launches));
    k_set_f32<<<g, 256, 0, st>>>(zout, w.c32, P, w.dsc);
    *launches += 2;
    return cudaGetLastError();
  };
  VMC_TRY(cudaMemsetAsync(x, 0, P * sizeof(double2), st));
  VMC_TRY(cudaMemcpyAsync(r, F, P * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  VMC_TRY(precondition(r, z));
  double rz = 0.0, f2 = 0.0;
  VMC_TRY(pcg_dots(r, z, P, w.scal_part, st, &rz, &f2));
  ++*launches;
  const double fn = std::sqrt(f2);
  VMC_TRY(cudaMemcpyAsync(p, z, P * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  double rel = fn > 0.0 ? 1.0 : 0.0;
  int it = 0;
  for (; it < std::max(1, maxit) && fn > 0.0; ++it) {
    VMC_TRY(apply(p, q));
    double pq = 0.0, dummy = 0.0;
    VMC_TRY(pcg_dots(p, q, P, w.scal_part, st, &pq, &dummy));
    if (!(pq > 0.0)) { rel = NAN; break; }
    const double alpha = rz / pq;
    k_pcg_update<<<g, 256, 0, st>>>(x, r, p, q, alpha, P);
    // the residual test first: the preconditioner (two triangular solves) is applied only
    // when another iteration follows
    double r2 = 0.0, r2b = 0.0;
    VMC_TRY(pcg_dots(r, r, P, w.scal_part, st, &r2, &r2b));
    *launches += 3;
    rel = std::sqrt(r2) / fn;
    if (!(rel == rel)) break;
    if (rel <= tol) { ++it; break; }
    VMC_TRY(precondition(r, z));
    double rz_new = 0.0;
    VMC_TRY(pcg_dots(r, z, P, w.scal_part, st, &rz_new, &r2b));
    ++*launches;
    const double beta = rz_new / rz;
    rz = rz_new;
    k_pcg_dir<<<g, 256, 0, st>>>(p, z, beta, P);
    ++*launches;
  }
  if (relres_rec) *relres_rec = rel;
  // explicit residual of the returned x with the operator itself
  double rel_ex = rel;
  if (fn > 0.0 && rel == rel) {
    VMC_TRY(apply(x, q));
    k_sub<<<g, 256, 0, st>>>(F, q, r, P);
    double d0 = 0.0, e2 = 0.0;
    VMC_TRY(pcg_dots(r, r, P, w.scal_part, st, &d0, &e2));
    *launches += 2;
    rel_ex = std::sqrt(e2) / fn;
  }
  if (iters) *iters = it;
  if (relres) *relres = rel_ex;
  return cudaGetLastError();
}

cudaError_t launch_update(double2* params, const double2* x, int64_t P, double dt,
                          cudaStream_t st) {
  k_update<<<grid_for(P, 256, 4096), 256, 0, st>>>(params, x, P, dt);
  return cudaGetLastError();
}

}  // namespace vmc
