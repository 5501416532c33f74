// vmc_internal.h -- structs and kernel launchers shared between the libvmc translation
// units.  Not part of the public ABI (that is include/vmc.h).
#pragma once
#include <algorithm>
#include <cstdint>
#include <functional>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace vmc {

// FP32 working copy of one lattice's RBM parameters (device pointers).
struct RbmDev {
  int N, M;
  const float2* a;    // [N]
  const float2* b;    // [M]
  const float2* Wt;   // [N][M]  (W transposed)
  // move tables: for move q (site q of a TFIM flip, bond q of a Heisenberg exchange) with
  // D_qk = 2 W_kq (flip) or 2 (W_ki - W_kj) (bond (i, j)): mth[q][k] = tanh D_qk and
  // mlc[q] = sum_k log cosh D_qk (real part, and imaginary part reduced to (-pi, pi]).  A
  // move with s_i changes theta_k by -s_i D_qk.
  const float2* mth;  // [moves][M]
  const float2* mlc;  // [moves]
  // mpre[2q + h] = exp(sum_k log cosh D_qk - da) with da = 2 s (a_i - a_j) for a bond (i, j),
  // 2 s a_q for a flip, s = +1 (h = 0) or -1 (h = 1): the factor of psi(s')/psi(s) that does
  // not depend on theta (rounded once from FP64)
  const float2* mpre; // [moves][2]
};

struct LatDev {
  int model;          // 0 TFIM, 1 Heisenberg
  int Lx, Ly, nb;
  float J, h;
};

struct SampleArgs {
  RbmDev rbm;
  LatDev lat;
  int8_t* chains;                 // [C][N] in/out
  int C;
  int L;                          // steps per sweep
  uint64_t seed, stream, sweep0;
  int n_therm, n_samples, sweeps_per_sample;
  int8_t* spins_out;              // [n_samples*C][N] or null
  float2* logpsi_out;             // [n_samples*C] or null
  float2* eloc_out;               // [n_samples*C] or null
  float2* t_out;                  // [n_samples*C][M] or null
  const float2* theta_in;         // [C][M] theta of the chains' current spins, or null
                                  // (then the kernel forms theta = b + W s itself)
  unsigned long long* n_accept;
  unsigned* status;
};

// ---- rbm.cu -------------------------------------------------------------------------
// move tables of the lattice's model from the FP64 parameters (computed in FP64)
cudaError_t launch_move_tables(const double2* p, int N, int M, int model, int Lx, int Ly,
                               float2* mth, float2* mlc, float2* mpre, cudaStream_t st);
cudaError_t launch_param_prep(const double2* p, int N, int M, float2* a, float2* b, float2* Wt,
                              cudaStream_t st);
cudaError_t launch_logpsi(const RbmDev& R, const int8_t* spins, int64_t n, float2* out,
                          unsigned* status, cudaStream_t st);
cudaError_t launch_eloc(const RbmDev& R, const LatDev& L, const int8_t* spins, int64_t n,
                        float2* out, unsigned* status, cudaStream_t st);
cudaError_t launch_theta_tanh(const RbmDev& R, const int8_t* spins, int64_t n, float2* T,
                              cudaStream_t st);
// theta[c][j] = b_j + sum_i W_ji s_ci for C configurations, as a tiled FP32 product with,
// per entry, the same fused multiply-adds in the same order (i = 0 .. N-1 from b_j) as the
// sampler's own per-chain formation, so the results are bit-identical to it
cudaError_t launch_theta_gemm(const RbmDev& R, const int8_t* spins, int64_t C, float2* theta,
                              cudaStream_t st);
// theta = b + W s of n configurations on the tensor cores (spins exact in BF16, W as a BF16
// hi/lo pair, FP32 accumulation); a wait that expires sets DEV_ERR_TIMEOUT in status
cudaError_t launch_theta_tc(const RbmDev& R, const int8_t* spins, int64_t n, float2* theta,
                            unsigned* status, cudaStream_t st);
cudaError_t launch_ok_dense(const int8_t* spins, const float2* T, int64_t n, int N, int M,
                            float2* O, cudaStream_t st);
cudaError_t launch_sample(const SampleArgs& A, cudaStream_t st);
// every chain of n_lat lattices in one persistent launch (lattice order `order`, heavy
// first; ustart[o] the first work unit of the o-th lattice, ustart[n_lat] the unit count)
// with mpl hidden slots per lane; the sweep counters in d_args_mut advance by `advance`
// afterwards (on the device)
cudaError_t launch_sample_batched(const SampleArgs* d_args, const int* d_order,
                                  const int* d_ustart, int n_lat, int Nmax, int mpl,
                                  unsigned* counter, int warps_per_block, int grid,
                                  uint64_t advance, SampleArgs* d_args_mut, cudaStream_t st);
int batched_blocks_per_sm(int mpl, int warps_per_block, int Nmax);
// chains of one lattice that share a warp in the batched sampler with mpl slots per lane
int batched_chains_per_warp(int M, int mpl);
// hidden slots per lane that the per-chain kernels use for M hidden units
int sample_slots_per_lane(int M);

// ---- sr.cu ----------------------------------------------------------------------------
// Energy statistics in FP64: out[0..3] = <E>.re, <E>.im, <|E-<E>|^2>, sqrt(var/n).
cudaError_t launch_estats(const float2* E, int64_t n, double* out, unsigned* status,
                          cudaStream_t st);

// Column sums of the log-derivatives and of the force in FP64:
//   meanO[k] = (1/n) sum_q O_qk,  F[k] = (1/n) sum_q conj(O_qk) (E_q - <E>),
// with O = [s | t | t (x) s] built on the fly from spins and T = tanh theta.
// partial: scratch of moments_partial_doubles(n, N, M) doubles.  One chunk of 1024 samples
// per grid z index, so n <= kMomentsMaxChunks * 1024.
static constexpr int64_t kMomentsMaxChunks = 65535;
int64_t moments_partial_doubles(int64_t n, int N, int M);
cudaError_t launch_moments(const int8_t* spins, const float2* T, const float2* E,
                           const double* estats, int64_t n, int N, int M, double* partial,
                           double2* meanO, double2* F, cudaStream_t st);

// Centred log-derivatives, transposed and split into real rows:
//   X[2k][q] = Re(O_qk - <O_k>), X[2k+1][q] = Im(...), zero padded to [rows_pad][ld].
// FP32 (X32) and/or the BF16 pair hi = bf16(x), lo = bf16(x - hi).
// mean2 [P] is a workspace (the mean as FP32 hi/lo pairs).
cudaError_t launch_build_x(const int8_t* spins, const float2* T, const double2* meanO,
                           float4* mean2, int64_t n, int N, int M, int64_t rows_pad, int64_t ld,
                           float* X32, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, __half* X16,
                           cudaStream_t st);

// S_kl = (1/n) sum_q conj(Xc_qk) Xc_ql from the real row Gram G = X X^T (FP32 SIMT):
//   S = (G_{2k,2l} + G_{2k+1,2l+1}) + i (G_{2k,2l+1} - G_{2k+1,2l}), written as double2
//   [P][P]; mirror = also write the upper triangle.
cudaError_t launch_gram_f32(const float* X, int64_t rows_pad, int64_t ld, int64_t P,
                            double inv_n, double2* S, bool mirror, float2* part,
                            int64_t part_cap, cudaStream_t st, bool real = false);

// Same contraction on the tensor cores (tcgen05, BF16 hi/lo split, FP32 accumulation
// in TMEM).  Returns cudaErrorNotSupported when the shapes are not supported.
// Optional outputs besides S (FP64, may be null): S2 = S as FP32 hi/lo pairs {hi.re,
// hi.im, lo.re, lo.im} (full matrix with the mirror), and Af = the FP32 input of the
// Cholesky factorisation (lower triangle, diagonal shifted by nu in shift_mode).
// lolo adds the fourth product lo.lo^T: S is then exactly the Gram of the BF16-rounded X
// (positive semi-definite up to FP32 accumulation), which the three-product split (lo.lo^T
// dropped, a PSD term) is not.
// part [part_cap float2] is a workspace: when the tiles alone cannot fill the GPU (small P)
// the sample range is split into chunks whose FP32 partial folds are summed in FP64.
cudaError_t launch_gram_tc(const __nv_bfloat16* Xhi, const __nv_bfloat16* Xlo,
                           int64_t rows_pad, int64_t ld, int64_t P, double inv_n, double2* S,
                           bool mirror, float4* S2, float2* Af, double nu, int shift_mode,
                           int prod, float2* part, int64_t part_cap, unsigned* status,
                           cudaStream_t st);
// split-K support shared by both Gram kernels: number of sample chunks for `tiles` lower
// tiles over nkb blocks of samples (>= 16 blocks a chunk, P*P*chunks <= part_cap), and the
// FP64 sum of the chunk partials part[c][k][l] (l <= k) into S / S2 / Af
int gram_kchunks(int64_t tiles, int nkb, int64_t P, int64_t part_cap);
cudaError_t launch_gram_reduce(const float2* part, int kchunks, int64_t P, double inv_n,
                               double2* S, float4* S2, float2* Af, double nu, int shift_mode,
                               bool mirror, cudaStream_t st);

// Schur-complement update of an FP32 complex Cholesky factor on the tensor cores:
// A[off+k][off+l] -= sum_m L_km conj(L_lm) for 0 <= l <= k < n, with L's panel given as
// real rows (row 2k = Re L_k., row 2k+1 = Im L_k.) split into BF16 hi/lo, K columns.
// A[off + k][off + l] -= (X X^H)_kl on l <= k < n from the BF16 hi/lo planes of X (real rows
// 2k, 2k + 1) (prod 3) or one FP16 plane (prod 1); the tiles of the first tail_cols complex
// columns are updated last.
cudaError_t launch_herk_tc(const __nv_bfloat16* Xhi, const __nv_bfloat16* Xlo, int64_t rows_pad,
                           int64_t K, int64_t n, float2* A32, int64_t ldA, int64_t off,
                           int tail_cols, int prod, unsigned* status, cudaStream_t st);

// ---- solve.cu -------------------------------------------------------------------------
struct SolveWork {
  int64_t P;
  double2* A64;    // [P][P] FP64 factor workspace (FP64 solver), may be null
  double2* D64;    // [ceil(P/64)][64][64] inverted diagonal blocks (FP64)
  float2* A32;     // [P][P] FP32 factor workspace (mixed solver), may be null
  float2* D32;     // inverted diagonal blocks (FP32)
  double2* r;      // [P] residual / forward-solve workspace
  double2* c;      // [P] right-hand side workspace
  float2* r32;     // [P]
  float2* y32;     // [P]
  float2* c32;     // [P]
  double* scal;    // [8] device scalars
  double* scal_part = nullptr;  // [256] block partials of the preconditioned CG's dots
  unsigned* bar;   // [128] the cooperative kernels' grid barrier, abort word and step counters
  double2* fin;    // [P] final right-hand sides of the triangular solves (float2 or double2 entries)
  float2 *T32f, *T32b;    // [ceil(P/256)][256][256] inverses of the 256-wide diagonal blocks
  double2 *T64f, *T64b;   //   (transposed for the forward solve; FP32 or FP64 solver)
  __nv_bfloat16* Xhi;  // panel operands of the tensor-core Schur updates
  __nv_bfloat16* Xlo;
  int64_t x_elems;     // capacity of Xhi / Xlo
  float4* S2;          // [P][P] S as FP32 hi/lo pairs (mixed solvers' residual)
  float* dsc;          // [P] equilibration scales of the mixed solvers' factor
  float4* x2;          // [P] iterate as FP32 hi/lo pairs
};

// Cholesky solve of (S + shift) x = F, FP64 throughout.
cudaError_t solve_cholesky_fp64(const double2* S, const double2* F, double2* x, double nu,
                                int mode, SolveWork& w, unsigned* status, cudaStream_t st,
                                int64_t* launches);
// Mixed solvers' inputs from an FP64 S: w.S2 (hi/lo pairs, full) and w.A32 (lower
// triangle + shift).  The tensor-core Gram writes both directly instead.
cudaError_t split_shift(const double2* S, double nu, int mode, SolveWork& w, cudaStream_t st);
// FP32 Cholesky of w.A32 + iterative refinement with residuals F - (S + shift) x formed from
// w.S2 in compensated FP32 arithmetic (hi/lo pairs, error-free products and sums);
// tc = trailing updates of 512-wide panels on the tensor cores (BF16 split) instead of
// FP32 SIMT.
cudaError_t solve_cholesky_mixed(const double2* F, double2* x, double nu, int mode, double tol,
                                 int maxit, bool tc, SolveWork& w, unsigned* status,
                                 cudaStream_t st, int64_t* launches, int* iters,
                                 double* relres);
// Preconditioned CG with an exactly applied operator y = A v (callback) and the FP32
// Cholesky factor of w.A32 (factored here; tensor-core Schur updates when tc) as the
// preconditioner; r, z, p, q are [P] work vectors.  Stops when the recursive residual is at
// most tol ||F|| (relres_rec) or after maxit iterations; relres is the explicit residual
// ||F - A x|| / ||F|| of the returned x.  Synchronises every iteration.
using PcgOperator = std::function<cudaError_t(const double2*, double2*)>;
cudaError_t solve_pcg_factor(const double2* F, double2* x, double tol, int maxit, bool tc,
                             const PcgOperator& apply, double2* r, double2* z, double2* p,
                             double2* q, SolveWork& w, unsigned* status, cudaStream_t st,
                             int64_t* launches, int* iters, double* relres, double* relres_rec);
// FP64 relative residual ||(S + shift) x - F|| / ||F|| (synchronises).
cudaError_t residual_fp64(const double2* S, const double2* F, const double2* x, double nu,
                          int mode, SolveWork& w, cudaStream_t st, double* relres);

// min(tiles, number of SMs), at least 1: the grid of the persistent tensor-core kernels
unsigned persistent_grid(int64_t tiles);

// CG operator products on the tensor cores (cg_tc.cu).  Shapes for N <= 256:
//   Sb [s_rows][kN] spins as BF16 (s_rows = n padded to 256), V planes [v_rows][kN] (rows
//   2j / 2j+1 = Re / Im V_j, 2M / 2M+1 = Re / Im v_a), Bs [b_rows][ldK] = spins^T;
//   out [kchunks][mtiles * 128][nbt * 128] and ybpart [kchunks][M] are the OhU partials.
struct CgTcShape {
  int64_t kN, s_rows, v_rows, ldK, b_rows;
  int nbt, mtiles, nkpc, kchunks;
  bool ok;
};
CgTcShape cg_tc_shape(int N, int M, int64_t n);
// u_q = sum_j t_qj (v_b,j + (Sb V^T)_qj) + (Sb V^T)_q,M - c; upart[b] = FP64 sum of u over
// CTA b's samples, *nup = number of CTAs
cudaError_t launch_cg_ov_tc(const __nv_bfloat16* Sb, const __nv_bfloat16* Vhi,
                            const __nv_bfloat16* Vlo, const CgTcShape& sh, const float2* T,
                            const float2* vb, const double* c, int M, int64_t n, float2* u,
                            double2* upart, int* nup, const int* done, unsigned* status,
                            cudaStream_t st);
// chunk partials of sum_q A_rq s_qi with A rows 2j / 2j+1 = Re / Im conj(t_qj) w_q, rows
// 2M / 2M+1 = Re / Im w_q, w = u - mean (mean: the two doubles at `mean` if not null, else
// the sum of the nup FP64 partials in upart over n), and of sum_q conj(t_qj) w_q.  u is read
// in whole 64-sample blocks (the buffer must be padded to a multiple of 64, finite).
cudaError_t launch_cg_ohu_tc(const __nv_bfloat16* Bs, const CgTcShape& sh, const float2* T,
                             const float2* u, const double2* upart, int nup, const double* mean,
                             int M, int64_t n, float* out, float2* ybpart, const int* done,
                             unsigned* status, cudaStream_t st);

// failure-path self-tests of the bounded waits (a flag / an mbarrier that nothing sets)
cudaError_t launch_selftest_flag_wait(unsigned* word2, unsigned* status, cudaStream_t st);
cudaError_t launch_selftest_mbar_wait(unsigned* status, cudaStream_t st);
cudaError_t launch_selftest_poll_wait(unsigned* word4, unsigned* status, cudaStream_t st);

// ---- cg.cu ----------------------------------------------------------------------------
struct CgProblem {
  const int8_t* spins;            // [n][N]
  const float2* T;                // [n][M] tanh theta
  int64_t n;
  int N, M;
  const double2* meanO;           // [P] <O>
  bool tc;                        // operator products on the tensor cores (BF16 split)
  unsigned* status;
};
constexpr int CG_VPART_DOUBLES = 2560;
constexpr int CG_T2_BLOCKS = 256;
struct CgWork {
  double2 *r, *p, *q, *y, *z;         // [P]
  double* D;                          // [P] shift diagonal
  double* Minv;                       // [P] inverse diagonal of S~ (preconditioner)
  double* t2;                         // [M]
  double* t2part;                     // [CG_T2_BLOCKS][M] partial sums of |t|^2
  float2 *va, *vb, *V;                // FP32 copies of the CG direction (vb: M + 128, the
                                      // tensor-core product copies 64-unit blocks)
  float2* u;                          // [n padded to 256] (the OhU kernel copies 64-sample blocks)
  float2* upart;                      // [ceil(M/64)][n]
  double* ustats;                     // [8]
  double* mpart;                      // moments scratch
  double* vpart;                      // [CG_VPART_DOUBLES] FP64 block partials of the CG sums
  double* sc;                         // [8] device scalars (|F|^2, |r|^2, <O>.p)
  int* flag;                          // [8] done, iterations performed; [4..7] stay zero
  float2* ones;                       // [n padded to 256] of (1, 0) (the <O> product's u)
  double* zero2;                      // [2] zeros (its mean)
  // tensor-core operator (capacities in elements; null when not allocated)
  __nv_bfloat16 *Sb, *Bs, *Vhi, *Vlo;
  float* part2;                       // OhU chunk partials
  float2* ybpart;                     // [kchunks][M]
  double2* ovpart;                    // [grid] FP64 sums of u per Ov CTA
  int64_t cap_sb, cap_bs, cap_v, cap_part2, cap_yb, cap_ov;
};
int64_t cg_partial_floats2(int64_t n, int M);
// diag(S) and the conjugated means; T and meanO must describe the sample set
cudaError_t cg_prepare(const CgProblem& pb, CgWork& w, double nu, int mode, cudaStream_t st,
                       int64_t* launches, bool operands_ready = false);
// <O> and F = <O^* (E - <E>)> (Eq. force_vector) with the tensor-core O^H u product
// (BF16 hi/lo operand, FP32 sums within K chunks, FP64 across); builds the spin operands
// the CG products use.  estats: FP64 <E> (re, im).  E: [n padded to 64] finite.
cudaError_t cg_moments_tc(const CgProblem& pb, const float2* E, const double* estats,
                          double2* meanO, double2* F, CgWork& w, cudaStream_t st,
                          int64_t* launches);
// a[k] = (1, 0) for k < n (default stream; the context's initialisation synchronises)
cudaError_t fill_ones(float2* a, int64_t n);
// y = S~ v once (after cg_prepare on the same problem)
cudaError_t cg_apply(const CgProblem& pb, CgWork& w, const double2* v, double2* y,
                     cudaStream_t st, int64_t* launches);
// CG on (1/n) Obar^H Obar + D from x0 = 0 until ||r|| <= tol ||F|| or maxit (synchronises
// once per iteration to read the residual)
cudaError_t cg_solve(const CgProblem& pb, const double2* F, double2* x, double tol, int maxit,
                     CgWork& w, cudaStream_t st, int64_t* launches, int* iters, double* relres);

// ---- tdvp.cu --------------------------------------------------------------------------
// Workspaces of the regularised TDVP right-hand side (P <= Pcap, n <= ncap samples).
struct TdvpWork {
  int64_t Pcap = 0, ncap = 0;
  int n_sm = 148;
  unsigned* status = nullptr;      // the context's status word
  double* w = nullptr;             // [ncap] sample weights (exact enumeration)
  float2* lp = nullptr;            // [ncap] log psi (exact enumeration)
  double* estats = nullptr;        // [8]
  double2* meanO = nullptr;        // [Pcap]
  double2* F = nullptr;            // [Pcap]
  double2* mom_part = nullptr;     // moments chunk partials
  int64_t mom_part_cap = 0;        // in double2
  double2* gram_part = nullptr;    // Gram chunk partials
  int64_t gram_part_cap = 0;       // in double2
  double2 *S = nullptr, *Q = nullptr, *A = nullptr, *V = nullptr, *S0 = nullptr;  // [Pcap]^2
  double* lam = nullptr;           // [Pcap] eigenvalues
  double2* rot = nullptr;          // [Pcap + 2] Jacobi rotations (c, sigma) per pair
  unsigned* bar = nullptr;         // grid barrier words [4]
  double* red = nullptr;           // [red_cap] per-block partials
  int red_cap = 0;
  double* info = nullptr;          // [2] Jacobi sweeps, relative off-diagonal norm
  double2* rho = nullptr;          // [Pcap] V^H F
  double* qd = nullptr;            // [Pcap] (V^H Q V)_kk
  double* lamp = nullptr;          // [Pcap] lambda^+
  double* lstats = nullptr;        // [4] lambda_1, lambda_min, kept components, min SNR
  double2* vec[8] = {};            // [Pcap] integrator vectors
  double* qpart = nullptr;         // [Pcap/256 + 1] quadratic-form partials
  // excited-state search (projected ansatz)
  float2* lp2 = nullptr;           // [ncap] log amplitudes of the reference state
  float2* e2 = nullptr;            // [ncap] local energies of the reference state
  float2* osc = nullptr;           // [ncap] 1 / (1 - rho) per sample
  float2* eexc = nullptr;          // [ncap] local energies of the projected ansatz
  double* wraw = nullptr;          // [ncap] unnormalised weights
  double* olap = nullptr;          // [8] overlap ratio lambda (see excited.cu)
};
int64_t tdvp_gram_chunks(int64_t n, int64_t P, int n_sm);
int64_t tdvp_gram_partial_doubles2(int64_t n, int64_t P, int n_sm);
cudaError_t launch_enum_states(int8_t* spins, int N, int64_t n, cudaStream_t st);
cudaError_t launch_born_weights(const float2* lp, int64_t n, double* w, unsigned* status,
                                cudaStream_t st);
// weighted <E> (tw.estats), <O> (tw.meanO) and F (tw.F); w = null: uniform 1/n (w must be
// normalised); osc = null or a per-sample complex factor multiplying every O_k(s); Od: a
// dense real O [n][Pd] (FP32) in place of the RBM's structured one (spins, T unused)
cudaError_t tdvp_moments(const int8_t* spins, const float2* T, const float2* E, const double* w,
                         const float2* osc, int64_t n, int N, int M, TdvpWork& tw,
                         cudaStream_t st, const float* Od = nullptr, int64_t Pd = 0);
// weighted S (tw.S) and energy-weighted Q (tw.Q), full Hermitian, FP64
cudaError_t tdvp_gram(const int8_t* spins, const float2* T, const float2* E, const double* w,
                      const float2* osc, int64_t n, int N, int M, TdvpWork& tw,
                      cudaStream_t st, const float* Od = nullptr, int64_t Pd = 0);
// w_out = w_in / sum(w_in); sums (may be null): sum w and sum w^2 of the input
cudaError_t launch_normalize_weights(const double* w_in, int64_t n, double* w_out,
                                     unsigned* status, cudaStream_t st, double* sums = nullptr);
// tw.S_kk *= 1 + nu
cudaError_t tdvp_shift(TdvpWork& tw, int64_t P, double nu, cudaStream_t st);
// tw.S = tw.V diag(tw.lam) tw.V^H (cooperative Jacobi on a copy in tw.A)
cudaError_t tdvp_eig(TdvpWork& tw, int64_t P, int max_sweeps, double tol, cudaStream_t st);
// out = -gamma V diag(lambda^+) V^H F
cudaError_t tdvp_solve(TdvpWork& tw, int64_t P, bool snr, double eps_pinv, int soft,
                       double eps_snr, double n_eff, double g_re, double g_im, double2* out,
                       cudaStream_t st);
// ---- excited.cu -----------------------------------------------------------------------
// overlap ratio lambda = exp(out[0]) (out[1] + i out[2]) from log amplitudes of psi and phi
// on samples of |phi|^2 (weights w or uniform)
cudaError_t launch_excited_lambda(const float2* lpsi, const float2* lphi, const double* w,
                                  int64_t n, double* out, unsigned* status, cudaStream_t st);
// per-sample 1/(1 - rho), unnormalised importance weights |1 - rho|^2 (x pw) and E_loc^Psi
cudaError_t launch_excited_prep(const float2* lpsi, const float2* lphi, const float2* epsi,
                                const float2* ephi, const double* pw, const double* olap,
                                int64_t n, float2* osc, double* wraw, float2* eexc,
                                cudaStream_t st);
cudaError_t launch_axpy2(const double2* y, double a, const double2* k1, double b, const double2* k2,
                         int64_t P, double2* out, cudaStream_t st);
cudaError_t launch_quad_form(const double2* S, const double2* x, const double2* y, int64_t P,
                             double* part, int* nparts, cudaStream_t st);

// ---- made.cu ---------------------------------------------------------------------------
struct MadeDev {
  int N, H;
  const float *W1, *b1, *W2, *b2, *W3, *b3;   // canonical layout (views into theta)
  const float *W1t, *W2t, *W3t;               // transposed copies
};
struct MadeWork {                             // batch workspaces, rows <= capacity
  float* logq;                                // [B]
  float *H1, *H2, *G1, *G2;                   // [B][H]
  float* G3;                                  // [B][N]
};
int64_t made_nparams(int N, int H);
MadeDev made_view(float* theta, float* W1t, float* W2t, float* W3t, int N, int H);
cudaError_t launch_made_transpose(const MadeDev& D, cudaStream_t st);
cudaError_t launch_made_logq(const MadeDev& D, const int8_t* spins, int64_t n, float* logq,
                             cudaStream_t st);
// gradient of -(1/n) sum log q over the batch into grad (canonical layout); w.logq holds log q
cudaError_t launch_made_grad(const MadeDev& D, const int8_t* spins, int64_t n, MadeWork& w,
                             float* grad, cudaStream_t st);
cudaError_t launch_adam(float* th, float* m, float* v, const float* g, int64_t np, int t, float lr,
                        cudaStream_t st);
// per-sample forward and backward of -log q(s) (no batch sum): w.logq, H1, H2, G1, G2, G3
cudaError_t launch_made_fwd_bwd(const MadeDev& D, const int8_t* spins, int64_t n, MadeWork& w,
                                cudaStream_t st);
cudaError_t launch_made_sample(const MadeDev& D, int64_t n, uint64_t seed, uint64_t stream,
                               uint64_t round, int8_t* spins, float* logq, cudaStream_t st);
cudaError_t launch_made_mh(int64_t C, int N, const int8_t* prop, const float2* prop_lp,
                           const float* prop_lq, int8_t* chains, float2* chain_lp,
                           float* chain_lq, uint64_t seed, uint64_t stream, uint64_t round,
                           unsigned long long* accepts, cudaStream_t st);

// theta <- theta - dt * x, then refresh the FP32 copies
cudaError_t launch_update(double2* params, const double2* x, int64_t P, double dt,
                          cudaStream_t st);

// ---- cnn.cu ---------------------------------------------------------------------------
// The translation-symmetric CNN-ELU ansatz (see cnn.cu).
struct CnnDev {
  int N, alpha;
  const float* W;   // [alpha][N]
  const float* b;   // [alpha]
};
struct CnnSampleArgs {
  CnnDev D;
  LatDev lat;
  int8_t* chains;                 // [C][N] in/out
  int64_t C;
  int L;                          // steps per sweep
  uint64_t seed, stream, sweep0;
  int n_therm, n_samples, sweeps_per_sample;
  int8_t* spins_out;              // [n_samples*C][N] or null
  float* logpsi_out;              // [n_samples*C] or null
  float2* eloc_out;               // [n_samples*C] or null
  unsigned long long* n_accept;
  unsigned* status;
};
cudaError_t launch_cnn_prep(const double* p, int alpha, int N, float* W, float* b, cudaStream_t st);
cudaError_t launch_cnn_sample(const CnnSampleArgs& A, cudaStream_t st);
cudaError_t launch_cnn_eval(const CnnDev& D, const LatDev& L, const int8_t* spins, int64_t n,
                            float* logpsi, float2* eloc, unsigned* status, cudaStream_t st);
// dense O [n][alpha (N + 1)] (FP32)
cudaError_t launch_cnn_ok(const CnnDev& D, const int8_t* spins, int64_t n, float* O, cudaStream_t st);
// theta += dt Re(thetadot)
cudaError_t launch_cnn_update(double* p, const double2* td, int64_t P, double dt, cudaStream_t st);

// ---- ar.cu ----------------------------------------------------------------------------
// The autoregressive network as the ansatz, psi = q^(1/2) (see ar.cu).
// configurations H connects each sample to: K = N (TFIM flips) or the bond count (Heisenberg
// exchanges; a parallel bond repeats the sample), out [n][K][N]
cudaError_t launch_ar_connected(const int8_t* spins, int64_t n, const LatDev& L, int8_t* out,
                                cudaStream_t st);
// E_loc(s) = diag + sum_k H_k exp((lq_k - lq) / 2) into E [n] (imaginary part 0)
cudaError_t launch_ar_eloc(const int8_t* spins, const float* lq, const float* lq_conn, int64_t n,
                           const LatDev& L, float2* E, unsigned* status, cudaStream_t st);
// <O_k> and F_k = <O_k (E - <E>)> (FP64, imaginary parts 0) from the per-sample backward in w
cudaError_t launch_ar_moments(const int8_t* spins, const MadeWork& w, const float2* E,
                              const double* estats, int64_t n, int N, int H, double* part,
                              int64_t part_cap, double2* meanO, double2* F, cudaStream_t st);
// X for the Gram in real rows: row k = O_k(q) - <O_k>, zero padded to [rows_pad][ld]
cudaError_t launch_ar_build_x(const int8_t* spins, const MadeWork& w, const double2* meanO,
                              int64_t n, int N, int H, int64_t rows_pad, int64_t ld, float* X,
                              cudaStream_t st);
// rows of S with a zero diagonal (masked weights, inactive units) become identity rows with
// F_k = 0, so that the solve leaves those parameters unchanged
cudaError_t launch_freeze_zero_rows(double2* S, double2* F, int64_t P, cudaStream_t st);
// theta_k -= dt Re x_k (FP64 master), then the FP32 copy
cudaError_t launch_ar_update(double* theta, const double2* x, int64_t P, double dt, float* theta32,
                             cudaStream_t st);
cudaError_t launch_to_f32(const double* a, int64_t n, float* b, cudaStream_t st);
cudaError_t launch_scale_f32(float* x, int64_t n, float a, cudaStream_t st);
// dense per-sample O [n][P] (FP32) from the per-sample backward in w
cudaError_t launch_ar_dense_o(const int8_t* spins, const MadeWork& w, int64_t n, int N, int H,
                              float* O, cudaStream_t st);


}  // namespace vmc
