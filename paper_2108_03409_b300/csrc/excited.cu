// excited.cu -- per-sample quantities of the excited-state search by projection
// (arXiv:2108.03409, section "Finding low-energy states", Eq. excited_state_ansatz):
//   Psi(s) = psi_theta(s) - lambda phi(s),  lambda = <psi / phi> over |phi|^2,
// with rho(s) = lambda phi(s) / psi(s):
//   Psi / psi = 1 - rho,  E_loc^Psi = (E_loc^psi - rho E_loc^phi) / (1 - rho),
//   O_k^Psi = O_k^psi / (1 - rho).
// Expectations under |Psi|^2 are taken over samples of |psi|^2 with the importance weights
// |1 - rho|^2 (times the Born weights of psi for exact enumeration).  FP64 arithmetic on the
// FP32 log amplitudes and local energies of both RBMs.
#include <cmath>

#include "vmc_device.cuh"
#include "vmc_internal.h"

namespace vmc {

namespace {

template <typename T>
__device__ __forceinline__ T bsum(T v, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  return r;
}

__device__ __forceinline__ double bmax(double v, double* sh) {
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

// lambda = exp(m) * mu, mu = sum_s w_s exp(d_s - m) (w = null: 1/n), d = log psi - log phi
// on samples of |phi|^2, m = max Re d.  out = {m, mu.re, mu.im}.  One block.
__global__ void k_excited_lambda(const float2* __restrict__ lpsi, const float2* __restrict__ lphi,
                                 const double* __restrict__ w, int64_t n, double* out,
                                 unsigned* status) {
  __shared__ double sh[32];
  double m = -INFINITY;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x)
    m = fmax(m, (double)lpsi[k].x - (double)lphi[k].x);
  m = bmax(m, sh);
  const double u = 1.0 / (double)n;
  double re = 0.0, im = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double dr = (double)lpsi[k].x - (double)lphi[k].x - m;
    const double di = (double)lpsi[k].y - (double)lphi[k].y;
    const double a = (w ? w[k] : u) * exp(dr);
    double sn, cs;
    sincos(di, &sn, &cs);
    re = fma(a, cs, re);
    im = fma(a, sn, im);
  }
  re = bsum(re, sh);
  im = bsum(im, sh);
  if (threadIdx.x == 0) {
    out[0] = m;
    out[1] = re;
    out[2] = im;
    if (!isfinite(m) || !isfinite(re) || !isfinite(im)) flag_error(status, DEV_ERR_NUMERIC);
  }
}

// per sample q of |psi|^2: rho = lambda phi / psi, the importance weight |1 - rho|^2 (times
// pw[q] if given), 1 / (1 - rho) and E_loc^Psi
__global__ void k_excited_prep(const float2* __restrict__ lpsi, const float2* __restrict__ lphi,
                               const float2* __restrict__ epsi, const float2* __restrict__ ephi,
                               const double* __restrict__ pw, const double* __restrict__ olap,
                               int64_t n, float2* __restrict__ osc, double* __restrict__ wraw,
                               float2* __restrict__ eexc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double m = olap[0], mr = olap[1], mi = olap[2];
  const double dr = (double)lphi[q].x - (double)lpsi[q].x + m;
  const double di = (double)lphi[q].y - (double)lpsi[q].y;
  const double a = exp(dr);
  double sn, cs;
  sincos(di, &sn, &cs);
  // rho = mu * exp(m + d)
  const double er = a * cs, ei = a * sn;
  const double rr = mr * er - mi * ei, ri = mr * ei + mi * er;
  const double ur = 1.0 - rr, ui = -ri;
  const double u2 = ur * ur + ui * ui;
  if (!(u2 > 0.0) || !isfinite(u2)) {
    osc[q] = make_float2(0.f, 0.f);
    wraw[q] = 0.0;
    eexc[q] = make_float2(0.f, 0.f);
    return;
  }
  const double inv = 1.0 / u2;
  const double cr = ur * inv, ci = -ui * inv;            // 1 / (1 - rho)
  const double2 ep = make_double2((double)epsi[q].x, (double)epsi[q].y);
  const double2 ef = make_double2((double)ephi[q].x, (double)ephi[q].y);
  const double nr = ep.x - (rr * ef.x - ri * ef.y), ni = ep.y - (rr * ef.y + ri * ef.x);
  osc[q] = make_float2((float)cr, (float)ci);
  wraw[q] = u2 * (pw ? pw[q] : 1.0);
  eexc[q] = make_float2((float)(nr * cr - ni * ci), (float)(nr * ci + ni * cr));
}

}  // namespace

cudaError_t launch_excited_lambda(const float2* lpsi, const float2* lphi, const double* w,
                                  int64_t n, double* out, unsigned* status, cudaStream_t st) {
  k_excited_lambda<<<1, 1024, 0, st>>>(lpsi, lphi, w, n, out, status);
  return cudaGetLastError();
}

cudaError_t launch_excited_prep(const float2* lpsi, const float2* lphi, const float2* epsi,
                                const float2* ephi, const double* pw, const double* olap,
                                int64_t n, float2* osc, double* wraw, float2* eexc,
                                cudaStream_t st) {
  k_excited_prep<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(lpsi, lphi, epsi, ephi, pw, olap, n,
                                                              osc, wraw, eexc);
  return cudaGetLastError();
}

}  // namespace vmc
