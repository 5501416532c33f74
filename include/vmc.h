/*
 * vmc.h -- C ABI of libvmc, the B300 (sm_103a) implementation of one NQS variational
 * Monte Carlo step for a complex RBM (arXiv:2108.03409, jVMC: section "Variational Monte
 * Carlo algorithms", Algorithm 1 "Single SR or TDVP time step").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Spins are int8 in {+1,-1}; s = +1 means Z = +1 (the paper's nets take 0/1 and map
 *    s = 2*s01 - 1, section "Variational wave functions").  A configuration is N
 *    consecutive bytes; batches are [n][N].
 *  - The RBM (Eq. rbm_ex) is read as theta_j = b_j + sum_i W_ji s_i,
 *    log psi(s) = sum_i a_i s_i + sum_j log cosh theta_j, with M = alpha*N hidden units.
 *  - Complex numbers are interleaved (re, im).  The parameter vector has
 *    P = N + M + N*M complex entries ordered [a(N) | b(M) | W(M x N, row-major W[j*N+i])];
 *    the log-derivatives O_k and the force F_k use the same order.
 *  - Lattices are Lx x Ly periodic, site i = x + Lx*y.  Bond b < N joins site b to its +x
 *    neighbour; bond b >= N (only when Ly > 1) joins site b-N to its +y neighbour.
 *  - "dev" pointers are CUDA device memory owned by the caller (e.g. torch tensors);
 *    "host" pointers are ordinary host memory.  The library never frees caller memory.
 *  - All device work is enqueued on the stream given to vmc_init.  Calls that return
 *    host results synchronise that stream; the others do not.
 *  - Errors: every call returns a vmc_status; no call aborts, asserts or traps.  Device
 *    errors (non-finite values, a non-positive Cholesky pivot, an expired bounded wait)
 *    are recorded in a device status word and reported by the next synchronising call.
 *    vmc_last_error() gives a message for the last failure on a context.
 *  - One context per host thread.
 */
#ifndef VMC_H
#define VMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VMC_OK = 0,
  VMC_ERR_ARG = 1,      /* invalid argument (NULL pointer, size out of range, bad index)   */
  VMC_ERR_CUDA = 2,     /* a CUDA runtime call failed                                      */
  VMC_ERR_OOM = 3,      /* device allocation failed at vmc_init                            */
  VMC_ERR_NUMERIC = 4,  /* NaN/Inf produced, Cholesky pivot <= 0, solver did not converge  */
  VMC_ERR_TIMEOUT = 5,  /* a bounded device-side wait expired                              */
  VMC_ERR_STATE = 6     /* call not valid in the context's current state                   */
} vmc_status;

enum { VMC_MODEL_TFIM = 0, VMC_MODEL_HEISENBERG = 1 };
enum { VMC_PREC_FP32 = 0, VMC_PREC_BF16SPLIT = 1 };
/* Solvers of S~ x = F: FP64 Cholesky; matrix-free CG; FP32 Cholesky + FP64 iterative
 * refinement; the same with the trailing (Schur) updates of 256-wide panels on the tensor
 * cores (BF16 hi/lo split) + FP64 iterative refinement. */
enum { VMC_SOLVER_CHOLESKY_FP64 = 0, VMC_SOLVER_CG = 1, VMC_SOLVER_CHOLESKY_MIXED = 2,
       VMC_SOLVER_CHOLESKY_TC = 3 };
enum { VMC_SHIFT_MULTIPLICATIVE = 0, VMC_SHIFT_ADDITIVE = 1 };

/* One lattice (Hamiltonian + RBM size).
 *  TFIM (section "Ground state search"; 2D form in "Unitary dynamics of pure states"):
 *      H = -J sum_<ij> Z_i Z_j - h sum_i X_i
 *  Heisenberg with Pauli matrices: H = J sum_<ij> (X_i X_j + Y_i Y_j + Z_i Z_j). */
typedef struct {
  int model;      /* VMC_MODEL_*                                   */
  int Lx, Ly;     /* Ly = 1 for a chain; N = Lx*Ly, 2 <= N <= 1024  */
  double J, h;
  int alpha;      /* M = alpha * N hidden units, M <= 512            */
} vmc_lattice;

/* Sampler and SR settings, shared by all lattices of a context. */
typedef struct {
  uint64_t seed;            /* Philox4x64-10 key word 0 (word 1 = lattice index)              */
  int n_chains;             /* Markov chains per lattice                                       */
  int sweep_len;            /* Metropolis steps per sweep; 0 means N                           */
  int therm_sweeps;         /* sweeps discarded before the first SR step                       */
  int sweeps_per_sample;    /* sweeps between two recorded samples of a chain (>= 1)           */
  int samples_per_chain;    /* samples per chain per SR step; Ns = n_chains * samples_per_chain */
  int precision;            /* VMC_PREC_*: arithmetic of the S = <O^H O>^c contraction         */
  int solver;               /* VMC_SOLVER_*                                                    */
  double shift;             /* diagonal shift nu (section "Diagonal shift")                     */
  int shift_mode;           /* VMC_SHIFT_*: (1+nu) S_kk (the paper's) or S_kk + nu             */
  int cg_maxit;             /* CG / refinement iteration cap                                   */
  double cg_tol;            /* relative residual target of the iterative solvers               */
  int made_hidden;          /* width H of the learned proposal's two hidden layers (multiple   */
                            /* of 32, <= 512); 0 = no learned proposal                         */
  int made_batch;           /* training batch of the learned proposal (0 = 4096)               */
  int tdvp;                 /* 1: allocate the TDVP workspaces (vmc_tdvp_rhs / vmc_tdvp_step;  */
                            /* every lattice's P <= 4096)                                      */
  int ar_ansatz;            /* 1: also allocate the workspaces of the autoregressive ansatz    */
                            /* (vmc_ar_*; needs made_hidden > 0 and a dense solver)            */
  int cnn_ansatz;           /* 1: also allocate the CNN-ELU ansatz (vmc_cnn_*; needs tdvp = 1; */
                            /* TFIM chains only, alpha = channels, alpha * N <= 512)          */
} vmc_config;

/* Statistics of one SR step (host struct filled by vmc_sr_step). */
typedef struct {
  double e_mean_re, e_mean_im;  /* <E_loc> over the Ns samples (Eq. Oloc_mean)              */
  double e_var;                 /* <|E_loc - <E>|^2>                                        */
  double e_stderr;              /* sqrt(e_var / Ns) (ignores autocorrelation)               */
  double acceptance;            /* accepted / proposed Metropolis steps in this step        */
  int64_t n_samples;            /* Ns                                                       */
  int solver_iters;             /* CG or refinement iterations (0 for the direct solve)     */
  double solver_relres;         /* ||S~ x - F|| / ||F|| of the returned update, FP64 (for    */
                                /* the BF16-split dense path: the preconditioned CG's own    */
                                /* recursive residual on the matrix-free FP32 operator)      */
  float ms_sample, ms_grad, ms_qfm, ms_solve, ms_update;  /* phase times (CUDA events)    */
  float ms_gram;                /* the S contraction kernel alone (CUDA events)             */
  int64_t launches;             /* kernels launched by this step                            */
  int solver_converged;         /* 1 if the solve reached cg_tol (the update was applied)   */
  double solver_relres_explicit; /* ||S~ x - F|| / ||F|| recomputed with the operator after  */
                                 /* an iterative solve (the recursive value is solver_relres) */
} vmc_sr_stats;

typedef struct vmc_ctx vmc_ctx;

/* Create a context for n_lattices lattices (1 <= n_lattices <= 4096).  Allocates every
 * device buffer the step needs (parameters, chains, samples, S or CG workspaces) once.
 * Parameters start at zero and chains at all-up; set them with vmc_set_params /
 * vmc_set_chains.  stream is a cudaStream_t (NULL = legacy default stream).
 * Returns VMC_ERR_ARG for invalid settings, VMC_ERR_OOM if the buffers do not fit. */
vmc_status vmc_init(const vmc_config* cfg, const vmc_lattice* lattices, int n_lattices,
                    void* stream, vmc_ctx** out);

/* Release every resource of the context.  NULL is ignored. */
void vmc_destroy(vmc_ctx* ctx);

/* Message for the last failure on ctx (static storage owned by ctx). */
const char* vmc_last_error(const vmc_ctx* ctx);

/* Copy the FP64 master parameters of one lattice in (host [P][2]) or out.  Setting
 * parameters also refreshes the FP32 working copies (section "Variational wave functions":
 * get/set_parameters). */
vmc_status vmc_set_params(vmc_ctx* ctx, int lattice, const double* params_host);
vmc_status vmc_get_params(vmc_ctx* ctx, int lattice, double* params_host);

/* Copy the chain states of one lattice in or out (host int8 [n_chains][N]).  Setting the
 * chains rewinds the sweep counter to 0 and re-arms thermalisation. */
vmc_status vmc_set_chains(vmc_ctx* ctx, int lattice, const int8_t* spins_host);
vmc_status vmc_get_chains(vmc_ctx* ctx, int lattice, int8_t* spins_host);

/* theta_j = b_j + sum_i W_ji s_i of the hidden units for a batch (Eq. rbm_ex; the chains'
 * theta cache at the start of a sampling run).  With VMC_PREC_BF16SPLIT the product runs on
 * the tensor cores: spins +-1 are exact in BF16, W enters as a BF16 hi + lo pair (2^-18
 * relative) and the sums accumulate in FP32; otherwise in FP32 on the SIMT cores (the FMA
 * chain of the sampler's own formation).  spins: dev int8 [n][N]; theta: dev float [n][M][2]
 * (interleaved Re, Im).  n = 0 is a no-op.  VMC_ERR_TIMEOUT if a tensor-core wait expired.
 * The sampler (vmc_sample, vmc_sr_step) starts its chains from this theta. */
vmc_status vmc_theta(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* theta);

/* log psi for a batch (Eq. rbm_ex; the __call__ of the NQS class).
 * spins: dev int8 [n][N]; logpsi: dev float [n][2].  n = 0 is a no-op.  The imaginary
 * part (the phase) is returned reduced to [-pi, pi]; so is the sampler's logpsi_out. */
vmc_status vmc_logpsi(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                      float* logpsi);

/* Local energy E_loc(s) = sum_s' H_ss' psi(s')/psi(s) (Eq. Oloc) for a batch, with every
 * psi(s')/psi(s) evaluated from the cached theta(s) of the sample (no s' is stored).
 * spins: dev int8 [n][N]; eloc: dev float [n][2]. */
vmc_status vmc_local_energy(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                            float* eloc);

/* Metropolis-Hastings sampling of |psi|^2 (sections "Quantum expectation values" and
 * "Sampler"): every chain of the lattice runs n_therm sweeps, then n_samples times
 * (sweeps_per_sample sweeps, record).  Step t of sweep k of chain c draws
 *   w = Philox4x64-10(counter = {c, k, t, 0}, key = {seed, lattice}),
 *   site/bond = floor((w0 >> 32) * K / 2^32), u = ((w1 >> 40) + 1/2) / 2^24,
 * proposes a single flip (TFIM, K = N) or the exchange of an anti-parallel nearest-
 * neighbour pair (Heisenberg, K = number of bonds; a parallel pair is a rejected no-op),
 * and accepts iff ln u < 2 Re[log psi(s') - log psi(s)].  The sweep counter k continues
 * across calls.  Outputs (dev, any may be NULL), sample index q = r * n_chains + c:
 *   spins_out [n_samples*n_chains][N] int8, logpsi_out and eloc_out [..][2] float. */
vmc_status vmc_sample(vmc_ctx* ctx, int lattice, int n_therm, int n_samples,
                      int8_t* spins_out, float* logpsi_out, float* eloc_out);

/* Log-derivatives and force for a given sample set (Eq. force_vector, section "Finding
 * low-energy states"): O_{a_i} = s_i, O_{b_j} = tanh theta_j, O_{W_ji} = tanh(theta_j) s_i;
 * F_k = <O_k^* E_loc> - <O_k^*><E_loc> with sample means.
 *   spins dev int8 [n][N], eloc dev float [n][2] (as from vmc_local_energy),
 *   O_out dev float [n][P][2] or NULL, F_out dev double [P][2] or NULL,
 *   E_stats host double [4] = (<E>.re, <E>.im, var, stderr) or NULL (synchronises).
 * n must not exceed the context's Ns. */
vmc_status vmc_grad(vmc_ctx* ctx, int lattice, const int8_t* spins, const float* eloc,
                    int64_t n, float* O_out, double* F_out, double* E_stats);

/* Quantum Fisher matrix S_kl = <O_k^* O_l> - <O_k^*><O_l> (Eq. qfm) of a sample set,
 * contracted with the given precision (VMC_PREC_*).  S_out: dev double [P][P][2], full
 * Hermitian matrix.  n must not exceed the context's Ns. */
vmc_status vmc_qfm(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, int precision,
                   double* S_out);

/* Regularised solve of S~ x = F (sections "Diagonal shift", Algorithm 1 line
 * "solve_TDVP_equation") with the context's shift, shift_mode and solver:
 *   S dev double [P][P][2] (Hermitian, read only), F dev double [P][2], x dev double [P][2].
 * iters/relres (host, may be NULL) report the iterative part.  Returns VMC_ERR_NUMERIC if
 * the factorisation meets a non-positive pivot or the iteration does not converge. */
vmc_status vmc_solve(vmc_ctx* ctx, int lattice, const double* S, const double* F, double* x,
                     int* iters, double* relres);

/* Matrix-free conjugate gradient for S~ x = F (section "Diagonal shift": the shift works
 * with iterative solvers) on the sample set `spins` (dev int8 [n][N], n <= Ns):
 *   S~ v = (1/n) Obar^H (Obar v) + D v,  D = shift * diag(S) (multiplicative) or shift,
 * with Obar v and Obar^H u evaluated from the RBM structure (O = [s | t | t (x) s]), never
 * forming S.  x0 = 0; stops when ||r|| <= cg_tol ||F|| or after cg_maxit iterations.
 * F, x: dev double [P][2].  iters / relres (host, may be NULL) report the finish
 * (relres is the recursively updated residual).  Synchronises once per iteration.
 * Returns VMC_ERR_NUMERIC if relres is still above cg_tol after cg_maxit iterations (x then
 * holds the last iterate, iters and relres are filled). */
vmc_status vmc_cg_solve(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                        const double* F, double* x, int* iters, double* relres);

/* One application y = S~ v of the operator vmc_cg_solve iterates with (same sample set
 * conventions, same arithmetic: the tensor-core products for VMC_PREC_BF16SPLIT contexts
 * with N <= 256, FP32 SIMT products otherwise).  v, y: dev double [P][2], v read only.
 * Only for contexts created for the CG solver. */
vmc_status vmc_sr_apply(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                        const double* v, double* y);

/* One full SR step (Algorithm 1, then the Euler update theta <- theta - dt x of
 * imaginary-time TDVP, Eq. stochastic_reconfiguration): sample Ns configurations, local
 * energies, log-derivatives, S and F, regularised solve, parameter update.  stats (host)
 * may be NULL.  Synchronises.  With the CG solver, a solve that does not reach cg_tol within
 * cg_maxit iterations returns VMC_ERR_NUMERIC without updating the parameters (the chains
 * have advanced; stats, if given, is filled with solver_converged = 0). */
vmc_status vmc_sr_step(vmc_ctx* ctx, int lattice, double dt, vmc_sr_stats* stats);

/* The same SR step on a given sample set instead of the chains' next samples (so that two
 * contexts, e.g. two precisions, can be compared on identical configurations): spins dev
 * int8 [n][N] with n = n_chains * samples_per_chain; E_loc and tanh(theta) are formed for
 * them, the chains do not move, acceptance is reported as 0.  VMC_ERR_ARG for another n;
 * otherwise as vmc_sr_step. */
vmc_status vmc_sr_step_on(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, double dt,
                          vmc_sr_stats* stats);

/* ---- learned proposal (masked autoregressive MLP; requires made_hidden > 0) -------------
 * q(s) = prod_d sigma(s_d z_d), z = W3 relu(W2 relu(W1 s + b1) + b2) + b3 with MADE masks
 * (Germain et al. 2015): hidden unit k has degree m(k) = (k mod (N-1)) + 1, W1[k][d] is used
 * iff m(k) >= d, W2[k2][k1] iff m(k2) >= m(k1), W3[d][k2] iff d > m(k2) (d 1-based).  It builds
 * on the paper's autoregressive factorisation (section "Autoregressive neural quantum
 * states") and is used as an independent Metropolis-Hastings proposal.  Parameters are
 * FP32 in the layout W1[H][N] | b1[H] | W2[H][H] | b2[H] | W3[N][H] | b3[N]. */
vmc_status vmc_made_set_params(vmc_ctx* ctx, int lattice, const float* params_host);
vmc_status vmc_made_get_params(vmc_ctx* ctx, int lattice, float* params_host);
/* log q(s) for a batch: spins dev int8 [n][N], logq dev float [n]; n <= max(n_chains, batch). */
vmc_status vmc_made_logq(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                         float* logq);
/* Gradient (dev float, parameter layout) of L = -(1/n) sum log q(s) over the batch; loss (host)
 * receives L.  Synchronises. */
vmc_status vmc_made_grad(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                         float* grad, double* loss);
/* Train q on samples (dev int8 [n][N]) by Adam (beta = 0.9, 0.999, eps = 1e-8, learning rate
 * lr) for `epochs` passes in consecutive batches of made_batch; loss (host) receives the mean
 * -log q over the samples after training.  Synchronises. */
vmc_status vmc_proposal_train(vmc_ctx* ctx, int lattice, const int8_t* samples, int64_t n,
                              int epochs, double lr, double* loss);
/* n exact draws from q (autoregressive): sample c of round r draws site d with
 * u = ((w[(d-1) mod 4] >> 40) + 1/2) / 2^24, w = Philox4x64-10({c, r, (d-1)/4, 2},
 * {seed, lattice}), s_d = +1 iff u < sigma(z_d).  spins dev int8 [n][N], logq dev float [n]
 * (may be NULL). */
vmc_status vmc_made_sample(vmc_ctx* ctx, int lattice, int64_t n, uint64_t round,
                           int8_t* spins, float* logq);
/* n_rounds rounds of independent Metropolis-Hastings on every chain: chain c draws s' from q
 * (round counter of the lattice) and accepts iff ln u < 2 Re[log psi(s') - log psi(s)] +
 * log q(s) - log q(s'), u from Philox4x64-10({c, r, 0, 3}, {seed, lattice}) word 1.  After each
 * round the chain states (spins_out [n_rounds*C][N]) and their local energies (eloc_out
 * [n_rounds*C][2]) are written (either may be NULL); acceptance (host) receives the
 * accepted fraction.  Synchronises. */
vmc_status vmc_sample_learned(vmc_ctx* ctx, int lattice, int n_rounds, int8_t* spins_out,
                              float* eloc_out, double* acceptance);

/* Every chain of every lattice in one persistent launch (batched sampling of many
 * independent lattices of uneven size; section "Batching for vectorization"): warps take
 * work units (the chains of one lattice that share a warp: a chain runs on a group of 4, 8,
 * 16 or 32 lanes, the fewest whose hidden slots per lane hold its M units) from an atomic
 * counter, the most expensive lattices first, and run the same sweeps, records and Philox
 * streams as vmc_sample does per lattice (n_therm sweeps, then n_samples records), so the
 * samples equal vmc_sample's.  Outputs (dev, may be NULL): spins_out holds lattice l's
 * samples [n_samples][n_chains][N_l] starting at byte n_samples * n_chains * (N_0 + ... +
 * N_{l-1}); eloc_out is [n_lattices][n_samples * n_chains][2].  The first call autotunes
 * the hidden slots per lane (the per-lattice kernels' width for the largest M, or a wider
 * instantiated width up to twice it and at most 8) and the warps per block of the
 * persistent grid (timed on one sweep, the faster of two launches each; chains restored).
 * use_graph = 1 captures the launch into a CUDA graph and replays it while
 * (n_therm, n_samples, spins_out, eloc_out) stay the same.  ms (host, may be NULL) receives
 * the device time of the call.  Synchronises. */
vmc_status vmc_sample_all(vmc_ctx* ctx, int n_therm, int n_samples, int8_t* spins_out,
                          float* eloc_out, int use_graph, double* ms);
/* Warps per block chosen by the autotuner (0 before the first vmc_sample_all). */
int vmc_autotuned_warps_per_block(const vmc_ctx* ctx);
/* Hidden slots per lane chosen by the autotuner (0 before the first vmc_sample_all). */
int vmc_autotuned_slots_per_lane(const vmc_ctx* ctx);

/* Checkpoint / resume.  vmc_get_state writes everything the method's trajectory depends on
 * into a host buffer: per lattice the FP64 parameters, the chains, the sweep counter (the
 * Philox counter of the local moves), the thermalised flag and, with a learned proposal,
 * its parameters, Adam moments, step and round counters (the seed is part of vmc_config).
 * With buf == NULL it only stores the required size in *len; otherwise *len (in: the
 * buffer's size) receives the bytes written.  vmc_set_state restores a state into a context
 * created with the same configuration and lattices (checked: VMC_ERR_ARG otherwise, the
 * context untouched); the continuation is then identical to the original's.  Both
 * synchronise. */
vmc_status vmc_get_state(vmc_ctx* ctx, void* buf, size_t* len);
vmc_status vmc_set_state(vmc_ctx* ctx, const void* buf, size_t len);

/* ---- TDVP: regularised right-hand side and adaptive Heun integrator --------------------
 * (sections "Unitary dynamics", "Regularization to invert the (quantum) Fisher matrix" and
 * "Utilities": TDVP, Stepper; requires a context created with tdvp = 1.)
 * The right-hand side solves Eq. tdvp_util with the identity for [[.]] (holomorphic RBM):
 *     S thetadot = -gamma F,  gamma = 1 (imaginary time: the SR step) or i (real time),
 * with S, F the connected correlators of Eq. qfm / Eq. force_vector over a weighted sample
 * set, computed in FP64 from the FP32 tanh(theta) and E_loc of the samples.  S (after the
 * optional multiplicative shift (1 + shift) S_kk) is diagonalised, S = V diag(lambda) V^H
 * (parallel cyclic Jacobi, FP64, to an off-diagonal norm of 1e-14 ||S||), rho = V^H F, and
 *     thetadot = -gamma V diag(lambda^+) rho,
 *     lambda^+_k = 1/lambda_k * d_pinv(|lambda_k / lambda_1|) * d_snr(SNR_k),
 * d_pinv = 1/(1 + (eps_pinv/r)^6) (soft) or [r >= eps_pinv] (hard, Eq. pinv_cutoff), 1 if
 * eps_pinv = 0 (then only lambda = 0 is dropped); d_snr = 1/(1 + (eps_snr/SNR)^6) with
 * SNR_k = |rho_k| / sqrt(var_s(rho_k(s)) / n), rho_k(s) = sum_l conj(V_lk) conj(Obar_l(s))
 * (E(s) - <E>), applied to Monte Carlo sample sets only (eps_snr = 0: off). */
typedef struct {
  double gamma_re, gamma_im;  /* gamma: (1, 0) imaginary time, (0, 1) real time             */
  double eps_pinv;            /* pseudo-inverse cutoff relative to lambda_1 (0 = none)     */
  int pinv_soft;              /* 1: soft cutoff, 0: hard cutoff (Eq. pinv_cutoff)          */
  double eps_snr;             /* SNR cutoff (0 = none)                                      */
  double shift;               /* multiplicative diagonal shift of S before the solve (>= 0) */
  int exact;                  /* vmc_tdvp_step / sample-less vmc_tdvp_rhs: 1 = exact sums   */
                              /* over all 2^N basis states (2^N <= Ns, N <= 24), Born weights */
  double eps_step;            /* vmc_tdvp_step: tolerance of the adaptive Heun step          */
  double tau_max;             /* vmc_tdvp_step: largest step size (0 = no limit)            */
  int max_retries;            /* vmc_tdvp_step: rejected attempts before giving up (0 = 50) */
  int jacobi_max_sweeps;      /* Jacobi sweep cap (0 = 40)                                  */
} vmc_tdvp_opts;

typedef struct {
  double e_mean_re, e_mean_im, e_var, e_stderr;  /* <E_loc> etc. at the (first) evaluation */
  double lam_max, lam_min;    /* lambda_1 = max |lambda| and the smallest eigenvalue of S   */
  int kept;                   /* eigen-components with damping factor >= 1/2                */
  double snr_min;             /* smallest SNR (0 when SNR damping is off)                   */
  int jacobi_sweeps;          /* sweeps the eigen-decomposition took                        */
  double jacobi_off;          /* its final off-diagonal norm relative to ||S||_F            */
  double tau_used, tau_next;  /* vmc_tdvp_step: accepted step size, proposed next one       */
  double delta;               /* vmc_tdvp_step: Fisher-norm difference of the two solutions */
  int retries;                /* vmc_tdvp_step: rejected attempts                            */
  int rhs_evals;              /* right-hand-side evaluations of the call                    */
  float ms;                   /* device time of the call (CUDA events)                      */
  float ms_gram, ms_eig;      /* the S/Q Gram and the eigen-decomposition of the first       */
                              /* evaluation (CUDA events)                                    */
} vmc_tdvp_stats;

/* thetadot of the current parameters on a sample set.  spins dev int8 [n][N] with
 * weights dev double [n] (normalised inside; NULL = uniform, i.e. Monte Carlo samples),
 * n <= Ns; or spins = NULL: the context makes the set itself, all 2^N basis states with
 * Born weights (opts->exact = 1) or Ns Metropolis samples of its chains (the chains
 * advance as in vmc_sr_step).  thetadot: dev double [P][2].  stats (host) may be NULL.
 * Synchronises.  Returns VMC_ERR_STATE without TDVP workspaces, VMC_ERR_NUMERIC for
 * non-finite results or a Jacobi iteration that did not converge. */
vmc_status vmc_tdvp_rhs(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                        const double* weights, const vmc_tdvp_opts* opts, double* thetadot,
                        vmc_tdvp_stats* stats);

/* One accepted step of the adaptive Heun integrator (section "Utilities", Stepper) on the
 * lattice's parameters y: with k1 = f(y, t), a Heun step of size tau,
 *     y_tau = y + tau/2 (k1 + f(y + tau k1)),
 * and two of size tau/2 (y_h = y + tau/4 (k1 + f(y + tau/2 k1)), then the same from y_h);
 * delta = ||y_tau - y_tau/2||_S with the Fisher norm ||v||_S = (1/P) sqrt(v^H S v), S taken
 * at y; tau <- tau (eps_step / delta)^(1/3) (capped at tau_max).  If delta <= eps_step the
 * two-half-step solution is kept and t advances by the step used, else the attempt is
 * repeated with the new tau (at most max_retries times; then the parameters are restored
 * and VMC_ERR_NUMERIC returned).  Every f evaluation is vmc_tdvp_rhs without spins.
 * t and tau (host, in/out): time and proposed step size.  Synchronises. */
vmc_status vmc_tdvp_step(vmc_ctx* ctx, int lattice, const vmc_tdvp_opts* opts, double* t,
                         double* tau, vmc_tdvp_stats* stats);

/* ---- excited states by projection (section "Finding low-energy states") ----------------
 * With a converged ground state phi on lattice ref_lattice (same model size, its parameters
 * fixed), the excited-state ansatz of `lattice` is Psi = psi - lambda phi (Eq.
 * excited_state_ansatz), lambda = <phi|psi>/<phi|phi> = <psi/phi> over |phi|^2.  With
 * rho(s) = lambda phi(s)/psi(s): E_loc^Psi = (E_loc^psi - rho E_loc^phi)/(1 - rho) (both with
 * the Hamiltonian of `lattice`), O^Psi_k = O^psi_k / (1 - rho).  Expectations under |Psi|^2
 * are taken over samples of |psi|^2 with importance weights |1 - rho|^2 (times the Born
 * weights of psi for exact sums).  Needs a context created with tdvp = 1. */
typedef struct {
  double lambda_re, lambda_im;  /* the overlap ratio used                                    */
  double ess;                   /* (sum w)^2 / sum w^2 of the importance weights              */
  vmc_tdvp_stats tdvp;          /* the right-hand side's statistics (energy of Psi, S, ...)   */
} vmc_excited_stats;

/* lambda from samples of |phi|^2: spins_phi dev int8 [n][N] (n <= Ns), or NULL: Ns
 * Metropolis samples of ref_lattice's chains (exact = 0) or all 2^N states with phi's Born
 * weights (exact = 1).  lambda_out host double [2].  Synchronises. */
vmc_status vmc_excited_lambda(vmc_ctx* ctx, int lattice, int ref_lattice, const int8_t* spins_phi,
                              int64_t n, int exact, double* lambda_out);
/* SR direction thetadot = -S^+ F of Psi (opts: gamma, shift, eps_pinv as for vmc_tdvp_rhs;
 * SNR damping is not applied to importance-weighted sets) on samples of |psi|^2: spins_psi
 * dev int8 [n][N] (n <= Ns), or NULL: Ns Metropolis samples of lattice's chains (opts->exact
 * = 0) or all basis states (opts->exact = 1).  lambda host double [2], or NULL for the last
 * value vmc_excited_lambda computed.  thetadot dev double [P][2]; stats may be NULL.
 * Synchronises. */
vmc_status vmc_excited_rhs(vmc_ctx* ctx, int lattice, int ref_lattice, const int8_t* spins_psi,
                           int64_t n, const double* lambda, const vmc_tdvp_opts* opts,
                           double* thetadot, vmc_excited_stats* stats);
/* One step of the search: lambda from fresh samples of |phi|^2 (or exact sums), then one
 * Euler step theta <- theta + dt thetadot with thetadot of vmc_excited_rhs (gamma = 1: SR). */
vmc_status vmc_excited_step(vmc_ctx* ctx, int lattice, int ref_lattice, double dt,
                            const vmc_tdvp_opts* opts, vmc_excited_stats* stats);

/* ---- the autoregressive network as the ansatz (section "Autoregressive neural quantum
 * states"; requires ar_ansatz = 1) --------------------------------------------------------
 * psi(s) = q(s)^(1/2) with q the masked autoregressive network described above for the
 * learned proposal (same layout and width made_hidden, its own FP64 master parameters):
 * q is normalised, so samples are exact independent draws (no Markov chain).  Real
 * parameters, real positive amplitudes; P = made parameter count (<= 16384).  The SR step is
 * real: O_k = (1/2) d log q / d theta_k, E_loc(s) = sum_s' H_ss' (q(s')/q(s))^(1/2),
 * theta <- theta - dt Re[(S + shift)^-1 F] with the context's dense solver; S is formed by
 * the FP32 SIMT Gram, and parameters whose S row is exactly zero (masked weights, inactive
 * units) are left unchanged. */
vmc_status vmc_ar_set_params(vmc_ctx* ctx, int lattice, const double* params_host);
vmc_status vmc_ar_get_params(vmc_ctx* ctx, int lattice, double* params_host);
/* log psi = (1/2) log q: spins dev int8 [n][N], logpsi dev float [n]. */
vmc_status vmc_ar_logpsi(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                         float* logpsi);
/* n exact draws (autoregressive sampling with the Philox stream of vmc_made_sample, round
 * counter of the lattice): spins_out dev int8 [n][N], logpsi_out dev float [n] (may be NULL). */
vmc_status vmc_ar_sample(vmc_ctx* ctx, int lattice, int64_t n, int8_t* spins_out,
                         float* logpsi_out);
/* E_loc for a batch (n <= Ns): eloc dev float [n][2] (imaginary part 0). */
vmc_status vmc_ar_local_energy(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                               float* eloc);
/* Per-sample O_k (O_out dev float [n][P] or NULL), <O_k> (meanO_out dev double [P] or NULL),
 * F_k = <O_k (E - <E>)> (F_out dev double [P] or NULL) and E_stats (host [4] or NULL) for a
 * batch (n <= Ns) with its local energies (dev float [n][2]).  Synchronises if E_stats. */
vmc_status vmc_ar_grad(vmc_ctx* ctx, int lattice, const int8_t* spins, const float* eloc,
                       int64_t n, float* O_out, double* meanO_out, double* F_out,
                       double* E_stats);
/* One SR step: Ns direct samples, E_loc, O, S (FP32 Gram, FP64 result), F, shifted solve,
 * Euler update.  stats as for vmc_sr_step (acceptance 1: every draw is new).  Synchronises. */
vmc_status vmc_ar_sr_step(vmc_ctx* ctx, int lattice, double dt, vmc_sr_stats* stats);

/* ---- the translation-symmetric CNN-ELU ansatz (section "Ground state search", Eq.
 * gs_nqs; requires cnn_ansatz = 1) ----------------------------------------------------------
 * log psi(s) = sum_{a < alpha} sum_r f_ELU(sum_l W_al s_{(l+r) mod N} + b_a) on a periodic
 * TFIM chain, alpha = the lattice's alpha (channels), real parameters [W (alpha x N) | b],
 * P = alpha (N + 1).  It uses the lattice's chains with its own sweep counter, the same
 * Philox stream and acceptance rule as vmc_sample (ln u < 2 [log psi(s') - log psi(s)]). */
vmc_status vmc_cnn_set_params(vmc_ctx* ctx, int lattice, const double* params_host);
vmc_status vmc_cnn_get_params(vmc_ctx* ctx, int lattice, double* params_host);
/* log psi (dev float [n], may be NULL) and E_loc (dev float [n][2], may be NULL) of a batch. */
vmc_status vmc_cnn_eval(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* logpsi,
                        float* eloc);
/* dense log-derivatives O [n][P] (dev float): O_{W_al} = sum_r f'(z_ar) s_{(l+r) mod N},
 * O_{b_a} = sum_r f'(z_ar). */
vmc_status vmc_cnn_grad(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* O_out);
/* Metropolis as vmc_sample (outputs dev, may be NULL: spins [n_samples*C][N], logpsi
 * [n_samples*C], eloc [n_samples*C][2]). */
vmc_status vmc_cnn_sample(vmc_ctx* ctx, int lattice, int n_therm, int n_samples, int8_t* spins_out,
                          float* logpsi_out, float* eloc_out);
/* One ground-state step of the paper's recipe: Ns samples, thetadot = -S^+ F from the FP64
 * TDVP core (opts: gamma = 1, the diagonal shift nu and the pseudo-inverse cutoff; the
 * caller lowers nu from step to step, e.g. nu = nu0 0.95^n), theta <- theta + dt thetadot. */
vmc_status vmc_cnn_sr_step(vmc_ctx* ctx, int lattice, double dt, const vmc_tdvp_opts* opts,
                           vmc_tdvp_stats* stats);

/* Failure-path self-test (no GPU fault): which = 0 runs the cooperative kernels' bounded
 * flag wait on a word that nothing sets, which = 1 the tensor-core kernels' bounded mbarrier
 * wait on a barrier that nothing arrives at, which = 2 the triangular solves' bounded poll
 * on a right-hand-side entry that nothing writes.  Each gives up after about 2e9 SM clock
 * cycles (about a second), records the expiry in the context's status word and returns:
 * the call returns VMC_ERR_TIMEOUT (the designed outcome) and the context stays usable.
 * Any other which: VMC_ERR_ARG.  Allocates a four-word scratch; synchronises. */
vmc_status vmc_selftest_wait_timeout(vmc_ctx* ctx, int which);

/* Number of kernel launches the library has issued on this context since it was created
 * (a counter kept by the host code). */
int64_t vmc_kernel_launches(const vmc_ctx* ctx);

/* Ns of the context (n_chains * samples_per_chain) and P of a lattice. */
int64_t vmc_num_samples(const vmc_ctx* ctx);
int64_t vmc_num_params(const vmc_ctx* ctx, int lattice);

/* The <O> / F reduction of vmc_grad without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc, for
 * example code running inside a framework that has already reserved the GPU's memory
 * for its own pool, or a step loop that must not allocate after start-up.  It needs no
 * context; the caller passes every input and output:
 *   spins      dev int8 [n][N]
 *   tanh_theta dev float [n][M][2]   (tanh theta_j of each sample, i.e. O_{b_j})
 *   eloc       dev float [n][2]
 *   F_out      dev double [P][2]     F_k = <O_k^* E_loc> - <O_k^*><E_loc>
 *   meanO_out  dev double [P][2] or NULL   <O_k>
 *   stream     cudaStream_t (NULL = legacy default stream); nothing is synchronised.
 * with P = N + M + N*M and the parameter order of this header.
 * Scratch: one file-scope device array of 2^21 doubles (16 MiB), held by a GPU from the
 * first call on it (or from library load with CUDA_MODULE_LOADING=EAGER) until the process
 * exits.  The call needs 8 + ceil(n/1024) * 4 * (M+1) * (N+1) doubles of it and returns
 * VMC_ERR_ARG when that exceeds the array (e.g. N = 64, M = 128 allows n <= 62 * 1024) or
 * when ceil(n/1024) > 65535 (one block column per 1024 samples).  It also returns
 * VMC_ERR_ARG for NULL inputs or sizes outside 1 <= N <= 1024, 1 <= M <= 512, n >= 1, and
 * VMC_ERR_CUDA if a launch fails.  Non-finite inputs give non-finite outputs (no status
 * word is kept).
 * The first call on a device looks up the array's device address with that device
 * current (a one-time set-up per device); make that first call before any stream
 * capture.  The address is kept for the life of the process: after a cudaDeviceReset
 * of that device this entry point must not be called again in the same process.  All
 * calls share the array and leave their partial sums in it: two calls whose work
 * overlaps on the GPU (different streams, no ordering) race on it. */
vmc_status vmc_force_noalloc(const int8_t* spins, const float* tanh_theta, const float* eloc,
                             int64_t n, int N, int M, double* F_out, double* meanO_out,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif /* VMC_H */
