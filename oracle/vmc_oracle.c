/*
 * vmc_oracle.c -- plain FP64 CPU oracle for one NQS variational Monte Carlo step
 * (arXiv:2108.03409, jVMC).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists so that the CUDA path can be checked
 * against slow, obviously correct definitions.  Only tests/, the package smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the CUDA library, and it never imports or calls it.
 *
 * Conventions (the paper's notation, with the readings stated here):
 *   - spins s_i in {+1,-1}, s_i = +1 <-> Z_i = +1 (the paper's 0/1 inputs map as s = 2*s01-1).
 *   - complex RBM (Eq. rbm_ex, section "Variational wave functions"), indices read as
 *       theta_j = b_j + sum_i W_ji s_i,   log psi(s) = sum_i a_i s_i + sum_j log cosh theta_j,
 *     j = 0..M-1 hidden, i = 0..N-1 visible.
 *   - parameter vector (complex, interleaved re/im doubles) ordered [a(N) | b(M) | W(M x N, row-major W[j*N+i])].
 *   - lattice: Lx x Ly periodic, site i = x + Lx*y; bond list = for each site its (x+1,y) bond,
 *     then (if Ly > 1) for each site its (x,y+1) bond.  A chain (Ly = 1) has N bonds, a square
 *     lattice 2N.
 *   - TFIM  (Examples section):  H = -J sum_<ij> Z_i Z_j - h sum_i X_i.
 *   - Heisenberg with Pauli matrices: H = J sum_<ij> (X_i X_j + Y_i Y_j + Z_i Z_j); its only
 *     off-diagonal element swaps an anti-parallel pair with amplitude 2J.
 *
 * Every entry point returns 0 on success, a nonzero code otherwise.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cd;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NUMERIC = 4 };
enum { MODEL_TFIM = 0, MODEL_HEIS = 1 };

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Counter-based RNG: Philox4x64-10 as defined by Salmon, Moraes, Dror, Shaw,            */
/* "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 64x64->128   */
/* multiplications with the published multipliers and Weyl key increments.              */
/* ------------------------------------------------------------------------------------ */
static void philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t mult0 = 0xD2E7470EE14C6C93ULL, mult1 = 0xCA5A826395121157ULL;
  const uint64_t weyl0 = 0x9E3779B97F4A7C15ULL, weyl1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    unsigned __int128 p0 = (unsigned __int128)mult0 * c0;
    unsigned __int128 p1 = (unsigned __int128)mult1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += weyl0; k1 += weyl1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

int orc_philox4x64(const uint64_t* ctr, const uint64_t* key, uint64_t* out) {
  if (!ctr || !key || !out) return ORC_ERR_ARG;
  philox4x64_10(ctr, key, out);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Lattice                                                                              */
/* ------------------------------------------------------------------------------------ */
static int n_bonds(int Lx, int Ly) { return (Ly > 1) ? 2 * Lx * Ly : Lx * Ly; }

static void bond_sites(int Lx, int Ly, int bond, int* i, int* j) {
  int N = Lx * Ly;
  int site = bond % N;
  int x = site % Lx, y = site / Lx;
  *i = site;
  if (bond < N) *j = ((x + 1) % Lx) + Lx * y;           /* horizontal */
  else          *j = x + Lx * ((y + 1) % Ly);           /* vertical   */
}

int orc_bonds(int Lx, int Ly, int* bi, int* bj) {
  if (Lx < 1 || Ly < 1 || !bi || !bj) return -1;
  int nb = n_bonds(Lx, Ly);
  for (int b = 0; b < nb; ++b) bond_sites(Lx, Ly, b, &bi[b], &bj[b]);
  return nb;
}

/* ------------------------------------------------------------------------------------ */
/* Complex RBM (Eq. rbm_ex)                                                              */
/* ------------------------------------------------------------------------------------ */

/* log cosh z evaluated without overflow: with z' = +-z chosen so that Re z' >= 0,
   cosh z = cosh z' = e^{z'} (1 + e^{-2z'}) / 2. */
static cd logcosh(cd z) {
  if (creal(z) < 0.0) z = -z;
  return z - M_LN2 + clog(1.0 + cexp(-2.0 * z));
}

static void rbm_theta(int N, int M, const cd* b, const cd* W, const int8_t* s, cd* theta) {
  for (int j = 0; j < M; ++j) {
    cd acc = b[j];
    for (int i = 0; i < N; ++i) acc += W[(size_t)j * N + i] * (double)s[i];
    theta[j] = acc;
  }
}

static cd rbm_logpsi(int N, int M, const cd* par, const int8_t* s, cd* theta_scratch) {
  const cd* a = par;
  const cd* b = par + N;
  const cd* W = par + N + M;
  rbm_theta(N, M, b, W, s, theta_scratch);
  cd acc = 0.0;
  for (int i = 0; i < N; ++i) acc += a[i] * (double)s[i];
  for (int j = 0; j < M; ++j) acc += logcosh(theta_scratch[j]);
  return acc;
}

/* log psi for a batch: out[n][2] = (re, im). */
/* theta_j = b_j + sum_i W_ji s_i of n configurations (Eq. rbm_ex), out: [n][M] complex. */
int orc_theta(int N, int M, const double* params, const int8_t* spins, int64_t n, double* out) {
  if (N < 1 || M < 1 || !params || (n > 0 && (!spins || !out))) return ORC_ERR_ARG;
  const cd* par = (const cd*)params;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k)
    rbm_theta(N, M, par + N, par + N + M, spins + k * N, (cd*)(out + 2 * k * M));
  return ORC_OK;
}

int orc_logpsi(int N, int M, const double* params, const int8_t* spins, int64_t n, double* out) {
  if (N < 1 || M < 1 || !params || (n > 0 && (!spins || !out))) return ORC_ERR_ARG;
  const cd* par = (const cd*)params;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t k = 0; k < n; ++k) {
    cd* th = (cd*)malloc(sizeof(cd) * (size_t)M);
    cd v = rbm_logpsi(N, M, par, spins + k * N, th);
    free(th);
    out[2 * k] = creal(v);
    out[2 * k + 1] = cimag(v);
    if (!isfinite(creal(v)) || !isfinite(cimag(v))) bad = 1;
  }
  return bad ? ORC_ERR_NUMERIC : ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Operator action s -> {s'_j}, {H_ss'_j}  (Eq. operator_mapping, "Operators" section)   */
/* Entry 0 is the diagonal element (s' = s).  Returns the number of entries.             */
/* ------------------------------------------------------------------------------------ */
static int connected(int model, int Lx, int Ly, double J, double h, const int8_t* s,
                     int8_t* sp, double* el) {
  int N = Lx * Ly, nb = n_bonds(Lx, Ly), cnt = 0;
  double diag = 0.0;
  for (int b = 0; b < nb; ++b) {
    int i, j;
    bond_sites(Lx, Ly, b, &i, &j);
    diag += (double)(s[i] * s[j]);
  }
  memcpy(sp, s, (size_t)N);
  el[0] = (model == MODEL_TFIM) ? -J * diag : J * diag;
  cnt = 1;
  if (model == MODEL_TFIM) {
    for (int i = 0; i < N; ++i) {           /* -h X_i flips site i */
      int8_t* t = sp + (size_t)cnt * N;
      memcpy(t, s, (size_t)N);
      t[i] = (int8_t)(-t[i]);
      el[cnt++] = -h;
    }
  } else {
    for (int b = 0; b < nb; ++b) {          /* J (XX + YY) swaps an anti-parallel pair, amplitude 2J */
      int i, j;
      bond_sites(Lx, Ly, b, &i, &j);
      if (s[i] == s[j]) continue;
      int8_t* t = sp + (size_t)cnt * N;
      memcpy(t, s, (size_t)N);
      t[i] = (int8_t)(-t[i]);
      t[j] = (int8_t)(-t[j]);
      el[cnt++] = 2.0 * J;
    }
  }
  return cnt;
}

static int max_connected(int model, int Lx, int Ly) {
  return 1 + ((model == MODEL_TFIM) ? Lx * Ly : n_bonds(Lx, Ly));
}

/* Connected configurations of one s (the get_s_primes interface for a single configuration).
   sp_out must hold max_connected*N bytes, el_out max_connected doubles. */
int orc_connected(int model, int Lx, int Ly, double J, double h, const int8_t* s,
                  int8_t* sp_out, double* el_out) {
  if (!s || !sp_out || !el_out || Lx < 1 || Ly < 1) return -1;
  return connected(model, Lx, Ly, J, h, s, sp_out, el_out);
}

int orc_max_connected(int model, int Lx, int Ly) { return max_connected(model, Lx, Ly); }

/* Local energy E_loc(s) = sum_s' H_ss' psi(s')/psi(s) (Eq. Oloc with O = H), where every
   log psi(s') is recomputed from scratch.  out[n][2]. */
int orc_eloc(int model, int Lx, int Ly, double J, double h, int M, const double* params,
             const int8_t* spins, int64_t n, double* out) {
  int N = Lx * Ly;
  if (N < 1 || M < 1 || !params || (n > 0 && (!spins || !out))) return ORC_ERR_ARG;
  if (model != MODEL_TFIM && model != MODEL_HEIS) return ORC_ERR_ARG;
  const cd* par = (const cd*)params;
  int mc = max_connected(model, Lx, Ly);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
  for (int64_t k = 0; k < n; ++k) {
    int8_t* sp = (int8_t*)malloc((size_t)mc * N);
    double* el = (double*)malloc(sizeof(double) * (size_t)mc);
    cd* th = (cd*)malloc(sizeof(cd) * (size_t)M);
    const int8_t* s = spins + k * N;
    int cnt = connected(model, Lx, Ly, J, h, s, sp, el);
    cd lp = rbm_logpsi(N, M, par, s, th);
    cd e = 0.0;
    for (int c = 0; c < cnt; ++c) {
      cd lpp = rbm_logpsi(N, M, par, sp + (size_t)c * N, th);
      e += el[c] * cexp(lpp - lp);
    }
    out[2 * k] = creal(e);
    out[2 * k + 1] = cimag(e);
    if (!isfinite(creal(e)) || !isfinite(cimag(e))) bad = 1;
    free(sp); free(el); free(th);
  }
  return bad ? ORC_ERR_NUMERIC : ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Log-derivatives O_k = d log psi / d theta_k (complex derivative of the holomorphic     */
/* RBM):  O_{a_i} = s_i,  O_{b_j} = tanh theta_j,  O_{W_ji} = tanh(theta_j) s_i.         */
/* out[n][P][2], P = N + M + N*M.                                                        */
/* ------------------------------------------------------------------------------------ */
int orc_ok(int N, int M, const double* params, const int8_t* spins, int64_t n, double* out) {
  if (N < 1 || M < 1 || !params || (n > 0 && (!spins || !out))) return ORC_ERR_ARG;
  const cd* par = (const cd*)params;
  const int64_t P = (int64_t)N + M + (int64_t)N * M;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) {
    cd* th = (cd*)malloc(sizeof(cd) * (size_t)M);
    const int8_t* s = spins + k * N;
    rbm_theta(N, M, par + N, par + N + M, s, th);
    cd* o = (cd*)(out + 2 * k * P);
    for (int i = 0; i < N; ++i) o[i] = (double)s[i];
    for (int j = 0; j < M; ++j) {
      cd t = ctanh(th[j]);
      o[N + j] = t;
      for (int i = 0; i < N; ++i) o[N + M + (int64_t)j * N + i] = t * (double)s[i];
    }
    free(th);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Quantum Fisher matrix and force vector (Eq. qfm, Eq. force_vector):                  */
/*   S_kl = <O_k^* O_l>^c,   F_k = <O_k^* E_loc>^c,   <AB>^c = <AB> - <A><B>,              */
/* with <.> the sample mean (Eq. Oloc_mean).  Two passes: means first, then centred       */
/* products (the same quantity, evaluated without cancellation).                         */
/* O[Ns][P][2], E[Ns][2] in; S[P][P][2], F[P][2], Emean[2] out.                          */
/* ------------------------------------------------------------------------------------ */
int orc_sr_matrices(int64_t Ns, int64_t P, const double* O, const double* E,
                    double* S, double* F, double* Emean) {
  if (Ns < 1 || P < 1 || !O || !E) return ORC_ERR_ARG;
  const cd* o = (const cd*)O;
  const cd* e = (const cd*)E;
  cd* mo = (cd*)calloc((size_t)P, sizeof(cd));
  cd me = 0.0;
  for (int64_t n = 0; n < Ns; ++n) me += e[n];
  me /= (double)Ns;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < P; ++k) {
    cd acc = 0.0;
    for (int64_t n = 0; n < Ns; ++n) acc += o[n * P + k];
    mo[k] = acc / (double)Ns;
  }
  if (Emean) { Emean[0] = creal(me); Emean[1] = cimag(me); }
  if (F) {
    cd* f = (cd*)F;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < P; ++k) {
      cd acc = 0.0;
      for (int64_t n = 0; n < Ns; ++n) acc += conj(o[n * P + k] - mo[k]) * (e[n] - me);
      f[k] = acc / (double)Ns;
    }
  }
  if (S) {
    cd* sm = (cd*)S;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < P; ++k) {
      for (int64_t l = 0; l < P; ++l) {
        cd acc = 0.0;
        for (int64_t n = 0; n < Ns; ++n) acc += conj(o[n * P + k] - mo[k]) * (o[n * P + l] - mo[l]);
        sm[k * P + l] = acc / (double)Ns;
      }
    }
  }
  free(mo);
  return ORC_OK;
}

/* Selected entries of S and F without storing the full matrix: S_{k,l} for the listed
   (k[q], l[q]) pairs and F_k for the listed fk[q].  Same definitions as orc_sr_matrices. */
int orc_sr_entries(int64_t Ns, int64_t P, const double* O, const double* E,
                   int64_t nq, const int64_t* kk, const int64_t* ll, double* s_out,
                   int64_t nf, const int64_t* fk, double* f_out) {
  if (Ns < 1 || P < 1 || !O || !E) return ORC_ERR_ARG;
  const cd* o = (const cd*)O;
  const cd* e = (const cd*)E;
  cd me = 0.0;
  for (int64_t n = 0; n < Ns; ++n) me += e[n];
  me /= (double)Ns;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nq; ++q) {
    int64_t k = kk[q], l = ll[q];
    cd mk = 0.0, ml = 0.0;
    for (int64_t n = 0; n < Ns; ++n) { mk += o[n * P + k]; ml += o[n * P + l]; }
    mk /= (double)Ns; ml /= (double)Ns;
    cd acc = 0.0;
    for (int64_t n = 0; n < Ns; ++n) acc += conj(o[n * P + k] - mk) * (o[n * P + l] - ml);
    acc /= (double)Ns;
    s_out[2 * q] = creal(acc);
    s_out[2 * q + 1] = cimag(acc);
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < nf; ++q) {
    int64_t k = fk[q];
    cd mk = 0.0;
    for (int64_t n = 0; n < Ns; ++n) mk += o[n * P + k];
    mk /= (double)Ns;
    cd acc = 0.0;
    for (int64_t n = 0; n < Ns; ++n) acc += conj(o[n * P + k] - mk) * (e[n] - me);
    acc /= (double)Ns;
    f_out[2 * q] = creal(acc);
    f_out[2 * q + 1] = cimag(acc);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Diagonal-shift regularisation ("Diagonal shift" subsection):                          */
/*   mode 0 (the paper's form): S~_kk' = (1 + nu delta_kk') S_kk'  -> S~_kk = (1+nu) S_kk */
/*   mode 1 (additive variant):  S~_kk = S_kk + nu                                        */
/* in place on S[P][P][2].                                                               */
/* ------------------------------------------------------------------------------------ */
int orc_shift(int64_t P, double* S, double nu, int mode) {
  if (P < 1 || !S || (mode != 0 && mode != 1)) return ORC_ERR_ARG;
  cd* s = (cd*)S;
  for (int64_t k = 0; k < P; ++k) {
    if (mode == 0) s[k * P + k] *= (1.0 + nu);
    else s[k * P + k] += nu;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Solve S~ x = F for Hermitian positive-definite S~ by the Cholesky factorisation        */
/* S~ = L L^H (L lower triangular, real positive diagonal) and two triangular solves,    */
/* all in FP64 complex.  S[P][P][2] is read (lower triangle used), x[P][2] written.       */
/* Returns ORC_ERR_NUMERIC if a pivot is not positive and finite.                        */
/* ------------------------------------------------------------------------------------ */
int orc_cholesky_solve(int64_t P, const double* S, const double* F, double* x) {
  if (P < 1 || !S || !F || !x) return ORC_ERR_ARG;
  const cd* a = (const cd*)S;
  cd* L = (cd*)calloc((size_t)(P * P), sizeof(cd));
  if (!L) return ORC_ERR_ARG;
  int rc = ORC_OK;
  for (int64_t j = 0; j < P && rc == ORC_OK; ++j) {
    double d = creal(a[j * P + j]);
    for (int64_t k = 0; k < j; ++k) d -= creal(L[j * P + k] * conj(L[j * P + k]));
    if (!(d > 0.0) || !isfinite(d)) { rc = ORC_ERR_NUMERIC; break; }
    double ljj = sqrt(d);
    L[j * P + j] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < P; ++i) {
      cd v = a[i * P + j];
      for (int64_t k = 0; k < j; ++k) v -= L[i * P + k] * conj(L[j * P + k]);
      L[i * P + j] = v / ljj;
    }
  }
  if (rc == ORC_OK) {
    const cd* f = (const cd*)F;
    cd* y = (cd*)malloc(sizeof(cd) * (size_t)P);
    for (int64_t i = 0; i < P; ++i) {            /* L y = F */
      cd v = f[i];
      for (int64_t k = 0; k < i; ++k) v -= L[i * P + k] * y[k];
      y[i] = v / L[i * P + i];
    }
    cd* xo = (cd*)x;
    for (int64_t i = P - 1; i >= 0; --i) {       /* L^H x = y */
      cd v = y[i];
      for (int64_t k = i + 1; k < P; ++k) v -= conj(L[k * P + i]) * xo[k];
      xo[i] = v / creal(L[i * P + i]);
    }
    free(y);
  }
  free(L);
  return rc;
}

/* ------------------------------------------------------------------------------------ */
/* The shifted Fisher matrix applied without storing it (Carleo & Troyer CG, "Diagonal    */
/* shift" subsection):                                                                    */
/*   S~ v = (1/Ns) Obar^H (Obar v) + D v,   Obar = O - <O>,  D = nu diag(S) (mode 0)     */
/*   or D = nu (mode 1).                                                                  */
/* sr_operator_setup forms <O> and D; sr_operator_apply forms q = S~ p (u: Ns scratch).   */
/* ------------------------------------------------------------------------------------ */
static void sr_operator_setup(int64_t Ns, int64_t P, const cd* o, double nu, int mode, cd* mo,
                              double* diag) {
  for (int64_t k = 0; k < P; ++k) {
    cd acc = 0.0;
    for (int64_t n = 0; n < Ns; ++n) acc += o[n * P + k];
    mo[k] = acc / (double)Ns;
  }
  for (int64_t k = 0; k < P; ++k) {
    double acc = 0.0;
    for (int64_t n = 0; n < Ns; ++n) { cd d = o[n * P + k] - mo[k]; acc += creal(d * conj(d)); }
    diag[k] = (mode == 0) ? nu * acc / (double)Ns : nu;
  }
}

static void sr_operator_apply(int64_t Ns, int64_t P, const cd* o, const cd* mo,
                              const double* diag, const cd* p, cd* u, cd* q) {
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < Ns; ++n) {
    cd acc = 0.0;
    for (int64_t k = 0; k < P; ++k) acc += (o[n * P + k] - mo[k]) * p[k];
    u[n] = acc;
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < P; ++k) {
    cd acc = 0.0;
    for (int64_t n = 0; n < Ns; ++n) acc += conj(o[n * P + k] - mo[k]) * u[n];
    q[k] = acc / (double)Ns + diag[k] * p[k];
  }
}

/* y = S~ v once.  O[Ns][P][2], v[P][2] in; y[P][2] out.                                 */
int orc_sr_apply(int64_t Ns, int64_t P, const double* O, double nu, int mode, const double* v,
                 double* y) {
  if (Ns < 1 || P < 1 || !O || !v || !y) return ORC_ERR_ARG;
  cd* mo = (cd*)calloc((size_t)P, sizeof(cd));
  double* diag = (double*)calloc((size_t)P, sizeof(double));
  cd* u = (cd*)malloc(sizeof(cd) * (size_t)Ns);
  sr_operator_setup(Ns, P, (const cd*)O, nu, mode, mo, diag);
  sr_operator_apply(Ns, P, (const cd*)O, mo, diag, (const cd*)v, u, (cd*)y);
  free(mo); free(diag); free(u);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Matrix-free conjugate gradient for S~ x = F with the operator above.  Plain CG, FP64,  */
/* x0 = 0; stops when ||r|| <= tol ||F||.                                                 */
/* O[Ns][P][2], F[P][2] in; x[P][2] out; *iters and *relres report the finish.           */
/* ------------------------------------------------------------------------------------ */
int orc_cg_solve(int64_t Ns, int64_t P, const double* O, const double* F, double nu, int mode,
                 double tol, int maxit, double* x, int* iters, double* relres) {
  if (Ns < 1 || P < 1 || !O || !F || !x) return ORC_ERR_ARG;
  const cd* o = (const cd*)O;
  const cd* f = (const cd*)F;
  cd* xo = (cd*)x;
  cd* mo = (cd*)calloc((size_t)P, sizeof(cd));
  double* diag = (double*)calloc((size_t)P, sizeof(double));
  cd* r = (cd*)malloc(sizeof(cd) * (size_t)P);
  cd* p = (cd*)malloc(sizeof(cd) * (size_t)P);
  cd* q = (cd*)malloc(sizeof(cd) * (size_t)P);
  cd* u = (cd*)malloc(sizeof(cd) * (size_t)Ns);
  sr_operator_setup(Ns, P, o, nu, mode, mo, diag);
  double fn = 0.0;
  for (int64_t k = 0; k < P; ++k) { xo[k] = 0.0; r[k] = f[k]; p[k] = f[k]; fn += creal(f[k] * conj(f[k])); }
  fn = sqrt(fn);
  double rr = fn * fn;
  int it = 0;
  while (it < maxit && sqrt(rr) > tol * fn) {
    sr_operator_apply(Ns, P, o, mo, diag, p, u, q);   /* q = S~ p */
    cd pq = 0.0;
    for (int64_t k = 0; k < P; ++k) pq += conj(p[k]) * q[k];
    double alpha = rr / creal(pq);
    double rr_new = 0.0;
    for (int64_t k = 0; k < P; ++k) {
      xo[k] += alpha * p[k];
      r[k] -= alpha * q[k];
      rr_new += creal(r[k] * conj(r[k]));
    }
    double beta = rr_new / rr;
    for (int64_t k = 0; k < P; ++k) p[k] = r[k] + beta * p[k];
    rr = rr_new;
    ++it;
  }
  if (iters) *iters = it;
  if (relres) *relres = (fn > 0) ? sqrt(rr) / fn : 0.0;
  free(mo); free(diag); free(r); free(p); free(q); free(u);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Update: the SR step is one Euler step of imaginary-time TDVP (section "Unitary         */
/* dynamics", last paragraph; Eq. stochastic_reconfiguration):  theta <- theta - dt * x. */
/* ------------------------------------------------------------------------------------ */
int orc_update(int64_t P, double* params, const double* x, double dt) {
  if (P < 1 || !params || !x) return ORC_ERR_ARG;
  for (int64_t k = 0; k < 2 * P; ++k) params[k] -= dt * x[k];
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Metropolis-Hastings sampling of p(s) = |psi(s)|^2 / <psi|psi> (section "Sampler",     */
/* section "Quantum expectation values"), many chains, each step of chain c in sweep k:  */
/*   w = Philox4x64-10(ctr = {c, k, step, 0}, key = {seed, stream})                       */
/*   idx = floor((w0 >> 32) * K / 2^32), K = N (TFIM site) or n_bonds (Heisenberg bond)  */
/*   u   = ((w1 >> 40) + 1/2) / 2^24                                                      */
/*   TFIM: s' = s with s_idx flipped.  Heisenberg: bond (i,j) = idx; if s_i == s_j the    */
/*   step is a rejected no-op, else s' = s with s_i and s_j swapped (Sz conserved).       */
/*   accept iff ln u < 2 Re[log psi(s') - log psi(s)]  (log psi recomputed from scratch).  */
/* One sweep = sweep_len steps (0 means N); after every sweep the state is recorded.      */
/* spins[C][N] in/out; rec[n_sweeps][C][N] (optional); min_margin[C] = smallest           */
/* |ln u - 2 Re dlogpsi| met by the chain (optional); n_acc[C] accepted moves (optional). */
/* ------------------------------------------------------------------------------------ */
int orc_metropolis(int model, int Lx, int Ly, int M, const double* params, int64_t C,
                   int8_t* spins, uint64_t seed, uint64_t stream, uint64_t chain0,
                   uint64_t sweep0, int n_sweeps, int sweep_len, int8_t* rec,
                   double* min_margin, int64_t* n_acc) {
  int N = Lx * Ly;
  if (N < 1 || M < 1 || !params || !spins || n_sweeps < 0) return ORC_ERR_ARG;
  if (model != MODEL_TFIM && model != MODEL_HEIS) return ORC_ERR_ARG;
  const cd* par = (const cd*)params;
  const int L = sweep_len > 0 ? sweep_len : N;
  const uint64_t K = (model == MODEL_TFIM) ? (uint64_t)N : (uint64_t)n_bonds(Lx, Ly);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t c = 0; c < C; ++c) {
    int8_t* s = spins + c * N;
    int8_t* sp = (int8_t*)malloc((size_t)N);
    cd* th = (cd*)malloc(sizeof(cd) * (size_t)M);
    double mm = INFINITY;
    int64_t acc = 0;
    cd lp = rbm_logpsi(N, M, par, s, th);
    for (int k = 0; k < n_sweeps; ++k) {
      for (int st = 0; st < L; ++st) {
        uint64_t ctr[4] = {chain0 + (uint64_t)c, sweep0 + (uint64_t)k, (uint64_t)st, 0};
        uint64_t key[2] = {seed, stream};
        uint64_t w[4];
        philox4x64_10(ctr, key, w);
        uint64_t idx = ((w[0] >> 32) * K) >> 32;
        double u = ((double)(w[1] >> 40) + 0.5) * 0x1.0p-24;
        memcpy(sp, s, (size_t)N);
        if (model == MODEL_TFIM) {
          sp[idx] = (int8_t)(-sp[idx]);
        } else {
          int i, j;
          bond_sites(Lx, Ly, (int)idx, &i, &j);
          if (s[i] == s[j]) continue;
          sp[i] = (int8_t)(-sp[i]);
          sp[j] = (int8_t)(-sp[j]);
        }
        cd lpp = rbm_logpsi(N, M, par, sp, th);
        double lhs = log(u), rhs = 2.0 * creal(lpp - lp);
        if (!isfinite(rhs)) bad = 1;
        double margin = fabs(lhs - rhs);
        if (margin < mm) mm = margin;
        if (lhs < rhs) {
          memcpy(s, sp, (size_t)N);
          lp = lpp;
          ++acc;
        }
      }
      if (rec) memcpy(rec + ((int64_t)k * C + c) * N, s, (size_t)N);
    }
    if (min_margin) min_margin[c] = mm;
    if (n_acc) n_acc[c] = acc;
    free(sp);
    free(th);
  }
  return bad ? ORC_ERR_NUMERIC : ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Masked autoregressive MLP proposal (MADE; Germain, Gregor, Murray, Larochelle 2015),   */
/* used as an independent Metropolis-Hastings proposal.  The paper's autoregressive      */
/* factorisation p(s) = p1(s1) p2(s2|s1) ... ("Autoregressive neural quantum states")      */
/* gives q(s) with exact sampling.                                                        */
/*   degrees (1-based): input d = 1..N; hidden k of both layers m(k) = (k mod (N-1)) + 1   */
/*   h1 = relu(W1 x + b1), W1[k][d] used iff m(k) >= d        (x_d = s_d)                 */
/*   h2 = relu(W2 h1 + b2), W2[k2][k1] used iff m(k2) >= m(k1)                             */
/*   z  = W3 h2 + b3,       W3[d][k2] used iff d > m(k2)                                   */
/*   q(s) = prod_d sigma(s_d z_d),  log sigma(x) = -log(1 + e^-x)                          */
/* parameters (doubles): W1[H][N] | b1[H] | W2[H][H] | b2[H] | W3[N][H] | b3[N].          */
/* ------------------------------------------------------------------------------------ */
static int made_deg(int k, int N) { return (N > 1) ? (k % (N - 1)) + 1 : 1; }

static double log_sigmoid(double x) {
  return (x >= 0.0) ? -log1p(exp(-x)) : x - log1p(exp(x));
}

int64_t orc_made_nparams(int N, int H) {
  return (int64_t)H * N + H + (int64_t)H * H + H + (int64_t)N * H + N;
}

typedef struct { const double *W1, *b1, *W2, *b2, *W3, *b3; } made_view;

static made_view made_split(const double* p, int N, int H) {
  made_view v;
  v.W1 = p;
  v.b1 = v.W1 + (int64_t)H * N;
  v.W2 = v.b1 + H;
  v.b2 = v.W2 + (int64_t)H * H;
  v.W3 = v.b2 + H;
  v.b3 = v.W3 + (int64_t)N * H;
  return v;
}

/* forward of one configuration; a1, a2 pre-activations [H], z logits [N]; returns log q */
static double made_fwd1(const made_view* v, int N, int H, const int8_t* s, double* a1, double* a2,
                        double* z) {
  for (int k = 0; k < H; ++k) {
    double acc = v->b1[k];
    const int mk = made_deg(k, N);
    for (int d = 1; d <= N; ++d)
      if (mk >= d) acc += v->W1[(int64_t)k * N + (d - 1)] * (double)s[d - 1];
    a1[k] = acc;
  }
  for (int k2 = 0; k2 < H; ++k2) {
    double acc = v->b2[k2];
    const int m2 = made_deg(k2, N);
    for (int k1 = 0; k1 < H; ++k1)
      if (m2 >= made_deg(k1, N) && a1[k1] > 0.0) acc += v->W2[(int64_t)k2 * H + k1] * a1[k1];
    a2[k2] = acc;
  }
  double lq = 0.0;
  for (int d = 1; d <= N; ++d) {
    double acc = v->b3[d - 1];
    for (int k2 = 0; k2 < H; ++k2)
      if (d > made_deg(k2, N) && a2[k2] > 0.0) acc += v->W3[(int64_t)(d - 1) * H + k2] * a2[k2];
    z[d - 1] = acc;
    lq += log_sigmoid((double)s[d - 1] * acc);
  }
  return lq;
}

/* log q(s) and the logits for a batch: logq[n], z[n][N] (z may be NULL) */
int orc_made_forward(int N, int H, const double* params, const int8_t* spins, int64_t n,
                     double* logq, double* z) {
  if (N < 2 || H < 1 || !params || (n > 0 && (!spins || !logq))) return ORC_ERR_ARG;
  made_view v = made_split(params, N, H);
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) {
    double* a1 = (double*)malloc(sizeof(double) * (size_t)(2 * H + N));
    double* a2 = a1 + H;
    double* zz = a2 + H;
    logq[q] = made_fwd1(&v, N, H, spins + q * N, a1, a2, zz);
    if (z) memcpy(z + q * N, zz, sizeof(double) * (size_t)N);
    free(a1);
  }
  return ORC_OK;
}

/* Gradient of the loss L = -(1/n) sum_q log q(s_q) (backpropagation through the masked
   layers; ReLU derivative 1 for a > 0).  grad has the parameter layout; returns L. */
int orc_made_grad(int N, int H, const double* params, const int8_t* spins, int64_t n,
                  double* grad, double* loss) {
  if (N < 2 || H < 1 || !params || !spins || !grad || n < 1) return ORC_ERR_ARG;
  const int64_t np = orc_made_nparams(N, H);
  made_view v = made_split(params, N, H);
  memset(grad, 0, sizeof(double) * (size_t)np);
  double* gW1 = grad;
  double* gb1 = gW1 + (int64_t)H * N;
  double* gW2 = gb1 + H;
  double* gb2 = gW2 + (int64_t)H * H;
  double* gW3 = gb2 + H;
  double* gb3 = gW3 + (int64_t)N * H;
  double* a1 = (double*)malloc(sizeof(double) * (size_t)(4 * H + 2 * N));
  double* a2 = a1 + H;
  double* z = a2 + H;
  double* g3 = z + N;
  double* g2 = g3 + N;
  double* g1 = g2 + H;
  double L = 0.0;
  for (int64_t q = 0; q < n; ++q) {
    const int8_t* s = spins + q * N;
    L -= made_fwd1(&v, N, H, s, a1, a2, z);
    /* d(-log sigma(s z))/dz = -s sigma(-s z) */
    for (int d = 0; d < N; ++d) {
      const double sd = (double)s[d];
      g3[d] = -sd / (1.0 + exp(sd * z[d])) / (double)n;
    }
    for (int k2 = 0; k2 < H; ++k2) g2[k2] = 0.0;
    for (int d = 1; d <= N; ++d) {
      gb3[d - 1] += g3[d - 1];
      for (int k2 = 0; k2 < H; ++k2) {
        if (!(d > made_deg(k2, N))) continue;
        const double h2 = a2[k2] > 0.0 ? a2[k2] : 0.0;
        gW3[(int64_t)(d - 1) * H + k2] += g3[d - 1] * h2;
        if (a2[k2] > 0.0) g2[k2] += v.W3[(int64_t)(d - 1) * H + k2] * g3[d - 1];
      }
    }
    for (int k1 = 0; k1 < H; ++k1) g1[k1] = 0.0;
    for (int k2 = 0; k2 < H; ++k2) {
      gb2[k2] += g2[k2];
      const int m2 = made_deg(k2, N);
      for (int k1 = 0; k1 < H; ++k1) {
        if (!(m2 >= made_deg(k1, N))) continue;
        const double h1 = a1[k1] > 0.0 ? a1[k1] : 0.0;
        gW2[(int64_t)k2 * H + k1] += g2[k2] * h1;
        if (a1[k1] > 0.0) g1[k1] += v.W2[(int64_t)k2 * H + k1] * g2[k2];
      }
    }
    for (int k1 = 0; k1 < H; ++k1) {
      gb1[k1] += g1[k1];
      const int m1 = made_deg(k1, N);
      for (int d = 1; d <= N; ++d)
        if (m1 >= d) gW1[(int64_t)k1 * N + (d - 1)] += g1[k1] * (double)s[d - 1];
    }
  }
  free(a1);
  if (loss) *loss = L / (double)n;
  return ORC_OK;
}

/* One Adam step (Kingma & Ba 2014): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
   theta <- theta - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps); t is 1-based. */
int orc_adam_step(int64_t np, double* theta, double* m, double* v, const double* g, int t,
                  double lr, double b1, double b2, double eps) {
  if (np < 1 || !theta || !m || !v || !g || t < 1) return ORC_ERR_ARG;
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t k = 0; k < np; ++k) {
    m[k] = b1 * m[k] + (1.0 - b1) * g[k];
    v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
    theta[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
  }
  return ORC_OK;
}

/* Autoregressive sampling of n configurations from q: site d of sample c in round r uses
   u = ((w[(d-1) mod 4] >> 40) + 1/2) / 2^24 from Philox4x64-10(ctr = {c, r, (d-1)/4, 2},
   key = {seed, stream}), and s_d = +1 iff u < sigma(z_d).  spins[n][N], logq[n]. */
int orc_made_sample(int N, int H, const double* params, int64_t n, uint64_t seed,
                    uint64_t stream, uint64_t round, int8_t* spins, double* logq,
                    double* min_margin) {
  if (N < 2 || H < 1 || !params || !spins) return ORC_ERR_ARG;
  made_view v = made_split(params, N, H);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    int8_t* s = spins + c * N;
    double* a1 = (double*)malloc(sizeof(double) * (size_t)(2 * H + N));
    double* a2 = a1 + H;
    double* z = a2 + H;
    double mm = INFINITY;
    for (int d = 0; d < N; ++d) s[d] = 1;
    for (int d = 1; d <= N; ++d) {
      /* logits of site d from the sites already drawn (later sites do not enter) */
      made_fwd1(&v, N, H, s, a1, a2, z);
      uint64_t ctr[4] = {(uint64_t)c, round, (uint64_t)((d - 1) / 4), 2};
      uint64_t key[2] = {seed, stream};
      uint64_t w[4];
      philox4x64_10(ctr, key, w);
      const double u = ((double)(w[(d - 1) % 4] >> 40) + 0.5) * 0x1.0p-24;
      const double p = 1.0 / (1.0 + exp(-z[d - 1]));
      const double margin = fabs(u - p);
      if (margin < mm) mm = margin;
      s[d - 1] = (u < p) ? 1 : -1;
    }
    if (logq) logq[c] = made_fwd1(&v, N, H, s, a1, a2, z);
    if (min_margin) min_margin[c] = mm;
    free(a1);
  }
  return ORC_OK;
}
