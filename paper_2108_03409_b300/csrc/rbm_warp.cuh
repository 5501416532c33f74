// rbm_warp.cuh -- warp-level building blocks of the complex-RBM kernels (shared by the
// evaluation, sampling and batched-sampling translation units).  A group of G lanes (the
// whole warp, G = 32, or an aligned quarter / eighth of it in the batched sampler) owns one
// configuration (or one chain); hidden unit j = glane + G*k lives in register slot k of
// group lane glane.  The group's reductions and broadcasts name only its own lanes.
#pragma once

#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

static constexpr unsigned FULL = 0xffffffffu;

// the lanes of this lane's group of G (G a power of two, at most 32)
template <int G>
__device__ __forceinline__ unsigned group_mask(int lane) {
  return G == 32 ? FULL : (((1u << (G & 31)) - 1u) << (lane & ~(G - 1)));
}

// xor-butterfly sums over a group (every lane of the group ends with the same bits)
template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gm, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ float group_sum_phase(float v, unsigned gm) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = wrap_phase(v + __shfl_xor_sync(gm, v, o));
  return v;
}

// theta_j = b_j + sum_i W_ji s_i for the warp's hidden slots, from spins in shared memory.
template <int MPL>
__device__ __forceinline__ void warp_theta(const RbmDev& R, const int8_t* s, int lane,
                                           float2 (&th)[MPL]) {
#pragma unroll
  for (int k = 0; k < MPL; ++k) {
    int hj = lane + 32 * k;
    th[k] = (hj < R.M) ? R.b[hj] : make_float2(0.f, 0.f);
  }
  for (int i = 0; i < R.N; ++i) {
    const float si = (float)s[i];
    const float2* w = R.Wt + (int64_t)i * R.M;
#pragma unroll
    for (int k = 0; k < MPL; ++k) {
      int hj = lane + 32 * k;
      if (hj < R.M) {
        float2 v = w[hj];
        th[k].x = fmaf(si, v.x, th[k].x);
        th[k].y = fmaf(si, v.y, th[k].y);
      }
    }
  }
}

// log psi = sum_i a_i s_i + sum_j log cosh theta_j (all lanes return the same value); the
// imaginary part is returned reduced to [-pi, pi] (a phase is defined mod 2 pi).
template <int MPL>
__device__ __forceinline__ float2 warp_logpsi(const RbmDev& R, const int8_t* s, int lane,
                                              const float2 (&th)[MPL]) {
  float re = 0.f, im = 0.f;
  for (int i = lane; i < R.N; i += 32) {
    float si = (float)s[i];
    re = fmaf(si, R.a[i].x, re);
    im = wrap_phase(fmaf(si, R.a[i].y, im));
  }
#pragma unroll
  for (int k = 0; k < MPL; ++k) {
    if (lane + 32 * k < R.M) {
      float2 lc = logcosh_c(th[k].x, th[k].y);
      re += lc.x;
      im = wrap_phase(im + lc.y);
    }
  }
  return make_float2(warp_sum(re), warp_sum_phase(im));
}

// A move q (a site flip, or a bond exchange of anti-parallel spins) with s_i the spin of
// its first site shifts theta_k by -s_i D_qk (D from the move tables):
//   cosh(theta - s_i D) / cosh(theta) = cosh D (1 - s_i t tanh D)      (t = tanh theta)
//   tanh(theta - s_i D) = (t - s_i tanh D) / (1 - s_i t tanh D)
// so a proposal reads one complex number per hidden unit (tanh D_qk) and adds the move's
// precomputed sum_k log cosh D_qk once.
__device__ __forceinline__ float2 move_factor(float2 t, float2 th, float si) {
  const float2 p = cmul(t, th);
  return make_float2(fmaf(-si, p.x, 1.f), -si * p.y);
}

// (the quotient with the hardware reciprocal, about 1 ulp: each accepted move adds a few
// units in the last place to t, and theta is recomputed from the spins periodically)
__device__ __forceinline__ float2 move_tanh_shift(float2 t, float2 th, float si) {
  const float2 td = make_float2(si * th.x, si * th.y);
  const float2 num = make_float2(t.x - td.x, t.y - td.y);
  const float2 tt = cmul(t, td);
  const float2 den = make_float2(1.0f - tt.x, -tt.y);
  const float inv = __fdividef(1.0f, fmaf(den.x, den.x, den.y * den.y));
  return make_float2(fmaf(num.x, den.x, num.y * den.y) * inv,
                     fmaf(num.y, den.x, -num.x * den.y) * inv);
}

// sum over the warp's hidden slots of log[cosh(theta_k - s_i D_qk) / cosh(theta_k)] for
// move q, as (log modulus, phase).  Each lane multiplies its factors and takes one log at
// the end; the running product is folded into the logs early only if it leaves
// [1e-15, 1e15] (checked every four factors).
template <int MPL, int G = 32>
__device__ __forceinline__ float2 warp_log_ratio(const RbmDev& R, int lane,
                                                 const float2 (&t)[MPL], int q, float si) {
  const int gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  float lr = 0.f, li = 0.f;
  float2 prod = make_float2(1.f, 0.f);
  const float2* row = R.mth + (int64_t)q * R.M;
#pragma unroll
  for (int k = 0; k < MPL; ++k) {
    int hj = gl + G * k;
    if (hj < R.M) prod = cmul(prod, move_factor(t[k], row[hj], si));
    if ((k & 3) == 3 && k != MPL - 1) {
      const float m2 = fmaf(prod.x, prod.x, prod.y * prod.y);
      if (m2 > 1e30f || m2 < 1e-30f) {
        lr += 0.5f * logf(m2);
        li += atan2f(prod.y, prod.x);
        prod = make_float2(1.f, 0.f);
      }
    }
  }
  lr += 0.5f * logf(fmaf(prod.x, prod.x, prod.y * prod.y));
  li += atan2f(prod.y, prod.x);
  const float2 c = R.mlc[q];
  return make_float2(group_sum<G>(lr, gm) + c.x, group_sum<G>(li, gm) + c.y);
}

// Complex product with both roundings of each part taken in a commutative order
// (products rounded, then added), so that the two partners of an xor butterfly level form
// the same bits.
__device__ __forceinline__ float2 cmul_sym(float2 a, float2 b) {
  return make_float2(__fsub_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)),
                     __fadd_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

// prod_k [1 - s_i t_k tanh D_qk] over all hidden units for move q, the same bits in every
// lane: each lane multiplies its own factors, an xor butterfly multiplies the lanes'.
template <int MPL, int G = 32>
__device__ __forceinline__ float2 warp_factor_prod(const RbmDev& R, int lane,
                                                   const float2 (&t)[MPL], int q, float si) {
  const int gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  float2 prod = make_float2(1.f, 0.f);
  const float2* row = R.mth + (int64_t)q * R.M;
#pragma unroll
  for (int k = 0; k < MPL; ++k) {
    const int hj = gl + G * k;
    if (hj < R.M) prod = cmul(prod, move_factor(t[k], row[hj], si));
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float2 p = make_float2(__shfl_xor_sync(gm, prod.x, o), __shfl_xor_sync(gm, prod.y, o));
    prod = cmul_sym(prod, p);
  }
  return prod;
}

// psi(s')/psi(s) for move q (a flip of site i, j < 0, or the exchange on bond (i, j)) with
// first-site spin si from the log-sum of its factors (group-wide): exp(sum_k log(1 - si t_k
// tanh D_qk) + sum_k log cosh D_qk - da), da = 2 si (a_i - a_j) or 2 si a_i.  No range limit.
template <int MPL, int G = 32>
__device__ __forceinline__ float2 warp_move_ratio_logsum(const RbmDev& R, int lane,
                                                         const float2 (&t)[MPL], int q,
                                                         float si, int i, int j) {
  const float2 lg = warp_log_ratio<MPL, G>(R, lane, t, q, si);
  float2 da = R.a[i];
  if (j >= 0) {
    da.x -= R.a[j].x;
    da.y -= R.a[j].y;
  }
  da = make_float2(2.f * si * da.x, 2.f * si * da.y);
  const float mag = expf(lg.x - da.x);
  float sn, cs;
  sincosf(lg.y - da.y, &sn, &cs);
  return make_float2(mag * cs, mag * sn);
}

// The same ratio as the factor product times the tabulated exp(sum_k log cosh D_qk - da),
// used while the product's squared modulus stays in [1e-30, 1e30] (every lane of the group
// holds the same product, so the branch is group-uniform); otherwise the log-sum form.
template <int MPL, int G = 32>
__device__ __forceinline__ float2 warp_move_ratio(const RbmDev& R, int lane,
                                                  const float2 (&t)[MPL], int q, float si,
                                                  int i, int j) {
  const float2 pr = warp_factor_prod<MPL, G>(R, lane, t, q, si);
  const float m2 = fmaf(pr.x, pr.x, pr.y * pr.y);
  if (m2 > 1e-30f && m2 < 1e30f) return cmul(pr, R.mpre[2 * q + (si < 0.f ? 1 : 0)]);
  return warp_move_ratio_logsum<MPL, G>(R, lane, t, q, si, i, j);
}

// Local-energy ratios of a lane group (G lanes, G <= 32), up to eloc_batch(G) moves at a
// time: group lane m holds move m (myq, first-site spin mysi, sites myi, myj; myj < 0 for a
// flip).  Each lane multiplies its own hidden slots' factors for every move (the table rows
// are read coalesced, as in a proposal), the partial products go through the group's part
// of the warp's shared-memory buffer eb, and lane m multiplies move m's G partials in lane
// order: no butterfly per move.  A move whose product leaves [1e-15, 1e15] in modulus takes
// the group-wide log-sum path.  Returns coef times this lane's move's ratio (0 for lanes
// >= nm).
static constexpr int kElocBatch = 16;
__host__ __device__ constexpr int eloc_batch(int G) { return G < kElocBatch ? G : kElocBatch; }
// float2 elements of one warp's buffer for groups of G lanes: 32 / G groups, eloc_batch(G)
// rows of G + 1 (padding against bank conflicts)
__host__ __device__ constexpr int eloc_buf_elems(int G) { return (32 / G) * eloc_batch(G) * (G + 1); }
__host__ __device__ constexpr int imax_c(int a, int b) { return a > b ? a : b; }
static constexpr int kElocBufBytes =
    8 * imax_c(imax_c(eloc_buf_elems(32), eloc_buf_elems(16)),
               imax_c(eloc_buf_elems(8), eloc_buf_elems(4)));

template <int MPL, int G>
__device__ __forceinline__ float2 warp_eloc_batch(const RbmDev& R, int lane,
                                                  const float2 (&t)[MPL], int nm, int myq,
                                                  float mysi, int myi, int myj, float coef,
                                                  float2* eb) {
  constexpr int LD = G + 1;
  const int gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  float2* ebg = eb + (lane / G) * (eloc_batch(G) * LD);
  for (int m = 0; m < nm; ++m) {
    const int q = __shfl_sync(gm, myq, m, G);
    const float si = __shfl_sync(gm, mysi, m, G);
    const float2* row = R.mth + (int64_t)q * R.M;
    float2 prod = make_float2(1.f, 0.f);
#pragma unroll
    for (int k = 0; k < MPL; ++k) {
      const int hj = gl + G * k;
      if (hj < R.M) prod = cmul(prod, move_factor(t[k], row[hj], si));
    }
    ebg[m * LD + gl] = prod;
  }
  __syncwarp(gm);
  float2 r = make_float2(0.f, 0.f);
  bool ok = true;
  if (gl < nm) {
    float2 p = ebg[gl * LD];
    for (int j = 1; j < G; ++j) p = cmul(p, ebg[gl * LD + j]);
    const float m2 = fmaf(p.x, p.x, p.y * p.y);
    ok = m2 > 1e-30f && m2 < 1e30f;
    if (ok) r = cmul(p, R.mpre[2 * myq + (mysi < 0.f ? 1 : 0)]);
  }
  __syncwarp(gm);                                       // ebg is rewritten by the next batch
  unsigned fb = __ballot_sync(gm, !ok);
  if (G < 32) fb = (fb >> (lane & ~(G - 1))) & ((1u << (G & 31)) - 1u);
  while (fb) {
    const int m = __ffs(fb) - 1;
    fb &= fb - 1;
    const float2 rr = warp_move_ratio_logsum<MPL, G>(
        R, lane, t, __shfl_sync(gm, myq, m, G), __shfl_sync(gm, mysi, m, G),
        __shfl_sync(gm, myi, m, G), __shfl_sync(gm, myj, m, G));
    if (gl == m) r = rr;
  }
  return make_float2(coef * r.x, coef * r.y);
}

// E_loc(s) = sum_s' H_ss' psi(s')/psi(s) from the cached t = tanh theta(s) (Eq. Oloc).
// The bonds are taken G at a time, one per lane of the chain's group: each lane finds its
// bond's sites and adds s_i s_j to the diagonal part; for the Heisenberg model a ballot then
// walks only the anti-parallel bonds, whose sites come from their lane by a shuffle.  With a
// ratio buffer eb the moves' ratios are formed in batches (warp_eloc_batch); without one,
// one at a time across the group (warp_move_ratio).
template <int MPL, int G = 32>
__device__ float2 warp_eloc(const RbmDev& R, const LatDev& L, const int8_t* s, int lane,
                            const float2 (&t)[MPL], float2* eb = nullptr) {
  if (eb) {                       // a ratio buffer: the moves' ratios in batches
    const int gl = lane & (G - 1);
    const unsigned gm = group_mask<G>(lane);
    constexpr int B = eloc_batch(G);
    float zz = 0.f;
    float2 acc = make_float2(0.f, 0.f);     // this lane's moves' contributions
    for (int b0 = 0; b0 < L.nb; b0 += G) {
      const int b = b0 + gl;
      int i = 0, j = 0;
      bool anti = false;
      if (b < L.nb) {
        bond_ends(L.Lx, L.Ly, b, &i, &j);
        zz += (float)(s[i] * s[j]);
        anti = s[i] != s[j];
      }
      if (L.model != 1) continue;
      const int ends = i | (j << 16);
      unsigned mask = __ballot_sync(gm, anti);
      if (G < 32) mask = (mask >> (lane & ~(G - 1))) & ((1u << (G & 31)) - 1u);
      while (mask) {                        // J(XX+YY): swap an anti-parallel pair, 2J
        int nm = 0, myq = 0, myi = 0, myj = 0;
        float mysi = 0.f;
        for (; nm < B && mask; ++nm) {
          const int src = __ffs(mask) - 1;
          mask &= mask - 1;
          const int pe = __shfl_sync(gm, ends, src, G);
          if (gl == nm) {
            myq = b0 + src;
            myi = pe & 0xffff;
            myj = pe >> 16;
            mysi = (float)s[myi];
          }
        }
        const float2 c = warp_eloc_batch<MPL, G>(R, lane, t, nm, myq, mysi, myi, myj,
                                                 2.f * L.J, eb);
        acc.x += c.x;
        acc.y += c.y;
      }
    }
    if (L.model == 0) {
      for (int i0 = 0; i0 < R.N; i0 += B) {   // -h X_i: flip site i
        const int nm = min(B, R.N - i0);
        const int myq = i0 + gl;
        const float mysi = (gl < nm) ? (float)s[myq] : 0.f;
        const float2 c = warp_eloc_batch<MPL, G>(R, lane, t, nm, myq, mysi, myq, -1, -L.h, eb);
        acc.x += c.x;
        acc.y += c.y;
      }
    }
    float2 e = make_float2(group_sum<G>(acc.x, gm), group_sum<G>(acc.y, gm));
    zz = group_sum<G>(zz, gm);
    e.x = fmaf(L.model == 0 ? -L.J : L.J, zz, e.x);
    return e;
  }
  const int gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  float zz = 0.f;                 // diagonal: sum over bonds of s_i s_j (exact small integers)
  float2 e = make_float2(0.f, 0.f);
  for (int b0 = 0; b0 < L.nb; b0 += G) {
    const int b = b0 + gl;
    int i = 0, j = 0;
    bool anti = false;
    if (b < L.nb) {
      bond_ends(L.Lx, L.Ly, b, &i, &j);
      zz += (float)(s[i] * s[j]);
      anti = s[i] != s[j];
    }
    if (L.model != 1) continue;
    const int ends = i | (j << 16);
    unsigned mask = __ballot_sync(gm, anti);
    if (G < 32) mask = (mask >> (lane & ~(G - 1))) & ((1u << (G & 31)) - 1u);
    while (mask) {                          // J(XX+YY): swap an anti-parallel pair, 2J
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const int pe = __shfl_sync(gm, ends, src, G);
      const int bi = pe & 0xffff, bj = pe >> 16;
      const float si = (float)s[bi];
      const float2 r = warp_move_ratio<MPL, G>(R, lane, t, b0 + src, si, bi, bj);
      e.x = fmaf(2.f * L.J, r.x, e.x);
      e.y = fmaf(2.f * L.J, r.y, e.y);
    }
  }
  zz = group_sum<G>(zz, gm);
  if (L.model == 0) {
    for (int i = 0; i < R.N; ++i) {           // -h X_i: flip site i
      const float si = (float)s[i];
      const float2 r = warp_move_ratio<MPL, G>(R, lane, t, i, si, i, -1);
      e.x = fmaf(-L.h, r.x, e.x);
      e.y = fmaf(-L.h, r.y, e.y);
    }
    e.x = fmaf(-L.J, zz, e.x);
  } else {
    e.x = fmaf(L.J, zz, e.x);
  }
  return e;
}

// ---------------------------------------------------------------------------------------
// a3/a4 + a6 (+ the t factors of a7): Metropolis sweeps with t = tanh theta cached in
// registers.  One warp per chain.  For a proposal s -> s' that changes theta by -d_k
// (d_k = 2 s_i W_ki, plus 2 s_j W_kj for an exchange),
//   psi(s')/psi(s) = exp(a-term) * prod_k cosh d_k * prod_k [1 - t_k tanh d_k],
// and the acceptance needs only its modulus squared.  On acceptance
// t_k <- tanh(theta_k - d_k) = (t_k - tanh d_k) / (1 - t_k tanh d_k).  Random numbers for
// 32 consecutive steps are drawn in parallel (lane q draws step t0+q and, for a bond
// exchange, finds the bond's two sites) and broadcast.  At
// record points the sample's spins, log psi, E_loc (fused, from the cached t) and t are
// written.  theta is recomputed from the spins (which removes the rounding drift of the
// t updates) at the start, at a record point where log psi is wanted, and at a record
// point after kResyncAccepts accepted moves since the last recomputation (each update
// adds a few units in the last place to t, so the drift stays near 1e-6 relative).
// ---------------------------------------------------------------------------------------
static constexpr int kResyncAccepts = 128;

template <int MPL, int G = 32>
__device__ __forceinline__ float2 warp_resync(const RbmDev& R, const int8_t* s, int lane,
                                              float2 (&t)[MPL], bool want_logpsi) {
  const int gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  float lr = 0.f, li = 0.f;
#pragma unroll
  for (int k = 0; k < MPL; ++k) {
    const int hj = gl + G * k;
    t[k] = make_float2(0.f, 0.f);
    if (hj < R.M) {
      float2 th = R.b[hj];
      for (int i = 0; i < R.N; ++i) {
        const float si = (float)s[i];
        const float2 v = R.Wt[(int64_t)i * R.M + hj];
        th.x = fmaf(si, v.x, th.x);
        th.y = fmaf(si, v.y, th.y);
      }
      t[k] = tanh_c(th.x, th.y);
      if (want_logpsi) {
        const float2 lc = logcosh_c(th.x, th.y);
        lr += lc.x;
        li = wrap_phase(li + lc.y);
      }
    }
  }
  if (!want_logpsi) return make_float2(0.f, 0.f);
  for (int i = gl; i < R.N; i += G) {
    const float si = (float)s[i];
    lr = fmaf(si, R.a[i].x, lr);
    li = wrap_phase(fmaf(si, R.a[i].y, li));
  }
  return make_float2(group_sum<G>(lr, gm), group_sum_phase<G>(li, gm));
}

// All sweeps of one chain by its group of G lanes (the whole warp for G = 32); s is the
// group's shared-memory spin buffer.  Every collective names only the group's lanes, so the
// groups of a warp may take different branches (accept / reject).
template <int MPL, bool HEIS, int G = 32>
__device__ void run_chain(const SampleArgs& A, int chain, int8_t* s, int lane,
                          float2* eb = nullptr) {
  const RbmDev& R = A.rbm;
  const LatDev& L = A.lat;
  const int N = R.N, M = R.M;
  const int gl = lane & (G - 1);
  const unsigned gm = group_mask<G>(lane);
  for (int i = gl; i < N; i += G) s[i] = A.chains[(int64_t)chain * N + i];
  __syncwarp(gm);

  float2 t[MPL];
  if (A.theta_in) {
#pragma unroll
    for (int k = 0; k < MPL; ++k) {
      const int hj = gl + G * k;
      t[k] = make_float2(0.f, 0.f);
      if (hj < M) {
        const float2 th = A.theta_in[(int64_t)chain * M + hj];
        t[k] = tanh_c(th.x, th.y);
      }
    }
  } else {
    warp_resync<MPL, G>(R, s, lane, t, false);
  }

  const uint32_t K = HEIS ? (uint32_t)L.nb : (uint32_t)N;
  const int total = A.n_therm + A.n_samples * A.sweeps_per_sample;
  unsigned long long n_acc = 0;
  int since_resync = 0;
  bool bad = false;

  for (int sw = 0; sw < total; ++sw) {
    const uint64_t sweep_id = A.sweep0 + (uint64_t)sw;
    for (int t0 = 0; t0 < A.L; t0 += G) {
      uint32_t my_idx = 0;
      float my_logu = 0.f;
      int my_ends = 0;                            // a bond's sites i | j << 16
      if (t0 + gl < A.L) {
        u64x4 w = philox4x64_10((uint64_t)chain, sweep_id, (uint64_t)(t0 + gl), 0ull,
                                A.seed, A.stream);
        mh_draw(w, K, &my_idx, &my_logu);
        if (HEIS) {
          int bi, bj;
          bond_ends(L.Lx, L.Ly, (int)my_idx, &bi, &bj);
          my_ends = bi | (bj << 16);
        }
      }
      const int nstep = min(G, A.L - t0);
      for (int q = 0; q < nstep; ++q) {
        const int idx = (int)__shfl_sync(gm, my_idx, q, G);
        const float logu = __shfl_sync(gm, my_logu, q, G);
        int i = idx, j = 0;
        if (HEIS) {
          const int pe = __shfl_sync(gm, my_ends, q, G);
          i = pe & 0xffff;
          j = pe >> 16;
          if (s[i] == s[j]) continue;             // parallel pair: rejected no-op
        }
        const float si = (float)s[i];
        const float two_re_da = HEIS ? -4.f * si * (R.a[i].x - R.a[j].x) : -4.f * si * R.a[i].x;
        const int64_t qrow = (int64_t)idx * M;     // move index: the bond, or the site
        float lsum = 0.f, prod = 1.f;
#pragma unroll
        for (int k = 0; k < MPL; ++k) {
          const int hj = gl + G * k;
          if (hj < M) {
            const float2 r = move_factor(t[k], R.mth[qrow + hj], si);
            prod *= fmaf(r.x, r.x, r.y * r.y);
          }
          if ((k & 7) == 7 || k == MPL - 1) {   // (hardware logarithm: ~1e-6 absolute)
            lsum += __logf(prod);
            prod = 1.f;
          }
        }
        const float two_re_delta = group_sum<G>(lsum, gm) + 2.f * R.mlc[idx].x + two_re_da;
        if (logu < two_re_delta) {
#pragma unroll
          for (int k = 0; k < MPL; ++k) {
            const int hj = gl + G * k;
            if (hj < M) t[k] = move_tanh_shift(t[k], R.mth[qrow + hj], si);
          }
          __syncwarp(gm);
          if (gl == 0) {
            s[i] = (int8_t)(-s[i]);
            if (HEIS) s[j] = (int8_t)(-s[j]);
          }
          __syncwarp(gm);
          ++n_acc;
          ++since_resync;
        }
      }
    }
    const int after = sw + 1 - A.n_therm;
    if (after > 0 && after % A.sweeps_per_sample == 0) {
      const int64_t rec = after / A.sweeps_per_sample - 1;
      const int64_t qs = rec * A.C + chain;
      float2 lp = make_float2(0.f, 0.f);
      if (A.logpsi_out || since_resync >= kResyncAccepts) {
        lp = warp_resync<MPL, G>(R, s, lane, t, A.logpsi_out != nullptr);
        since_resync = 0;
      }
      if (A.t_out)
#pragma unroll
        for (int k = 0; k < MPL; ++k) {
          const int hj = gl + G * k;
          if (hj < M) A.t_out[qs * M + hj] = t[k];
        }
      if (A.spins_out)
        for (int i = gl; i < N; i += G) A.spins_out[qs * N + i] = s[i];
      if (A.logpsi_out) {
        if (gl == 0) A.logpsi_out[qs] = lp;
        bad |= !isfinite(lp.x) || !isfinite(lp.y);
      }
      if (A.eloc_out) {
        const float2 e = warp_eloc<MPL, G>(R, L, s, lane, t, eb);
        if (gl == 0) A.eloc_out[qs] = e;
        bad |= !isfinite(e.x) || !isfinite(e.y);
      }
    }
  }
  __syncwarp(gm);
  for (int i = gl; i < N; i += G) A.chains[(int64_t)chain * N + i] = s[i];
  if (gl == 0) {
    if (A.n_accept) atomicAdd(A.n_accept, n_acc);
    if (bad) flag_error(A.status, DEV_ERR_NUMERIC);
  }
}

// lanes per chain in the batched sampler: the smallest group of 4, 8, 16 or 32 lanes whose
// MPL slots per lane hold the lattice's M hidden units (several chains share a warp when
// M is small against the warp's 32 MPL slots)
__host__ __device__ constexpr int batched_group(int M, int mpl) {
  return M <= 4 * mpl ? 4 : M <= 8 * mpl ? 8 : M <= 16 * mpl ? 16 : 32;
}

// hidden slots per lane: ceil(M / 32) rounded up to one of the instantiated widths
// (at most a third of the lanes' slots idle, e.g. M = 288 -> 10 slots of 32)
static inline int pick_mpl(int M) {
  const int m = (M + 31) / 32;
  static const int widths[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};
  for (int w : widths)
    if (w >= m) return w;
  return 0;
}

#define VMC_MPL_CASE(V, ...) case V: { constexpr int MPL = V; __VA_ARGS__; } break;
#define VMC_DISPATCH_MPL(M, ...)                                                        \
  switch (pick_mpl(M)) {                                                                \
    VMC_MPL_CASE(1, __VA_ARGS__) VMC_MPL_CASE(2, __VA_ARGS__) VMC_MPL_CASE(3, __VA_ARGS__) \
    VMC_MPL_CASE(4, __VA_ARGS__) VMC_MPL_CASE(5, __VA_ARGS__) VMC_MPL_CASE(6, __VA_ARGS__) \
    VMC_MPL_CASE(8, __VA_ARGS__) VMC_MPL_CASE(10, __VA_ARGS__)                          \
    VMC_MPL_CASE(12, __VA_ARGS__) VMC_MPL_CASE(16, __VA_ARGS__)                         \
    default: return cudaErrorInvalidValue;                                              \
  }

static constexpr int kWarps = 4;
static constexpr int kMaxChainsPerWarp = 8;   // batched sampler: groups of 4 lanes

// resident 4-warp blocks per SM that the per-chain sampler kernels are compiled for (a
// register budget per thread of 64 / 72 / 80 / 96 by the hidden slots per lane)
__host__ __device__ constexpr int sample_min_blocks(int mpl) {
  return mpl <= 4 ? 8 : mpl <= 6 ? 7 : mpl <= 8 ? 6 : 5;
}

static inline size_t spin_smem(int N) { return (size_t)kWarps * ((N + 15) & ~15); }

// Dynamic shared memory of the 4-warp sampling / local-energy blocks: the warps' spin
// buffers, then one local-energy ratio buffer per warp (spin_smem is a multiple of 16).
static inline size_t sample_smem(int N) { return spin_smem(N) + (size_t)kWarps * kElocBufBytes; }
__device__ __forceinline__ float2* eloc_buffer(int8_t* sm, int N, int wib) {
  return reinterpret_cast<float2*>(sm + kWarps * ((N + 15) & ~15) + wib * kElocBufBytes);
}

}  // namespace vmc
