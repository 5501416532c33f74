// api.cu -- the extern "C" entry points of libvmc (declared in include/vmc.h): context
// life cycle, parameter and chain transfer, and the steps of Algorithm 1 (sample,
// evaluate, gradients, local energies, S and F, solve) followed by the Euler update.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vmc.h"
#include "vmc_device.cuh"
#include "vmc_internal.h"

using namespace vmc;

namespace {

struct LatticeState {
  vmc_lattice lat;
  int N, M, nb;
  int64_t P;
  double2* params = nullptr;   // FP64 master [P]
  float2* a = nullptr;         // FP32 copies
  float2* b = nullptr;
  float2* Wt = nullptr;
  float2* mth = nullptr;       // move tables (tanh of the move's theta shift | sum of log cosh)
  float2* mlc = nullptr;
  int8_t* chains = nullptr;    // [C][N]
  uint64_t sweep = 0;          // sweeps done by every chain
  bool thermalized = false;
  // learned proposal (MADE)
  float* made = nullptr;       // FP32 parameters, canonical layout
  float *made_m = nullptr, *made_v = nullptr, *made_g = nullptr;
  float *W1t = nullptr, *W2t = nullptr, *W3t = nullptr;
  int made_t = 0;              // Adam step counter
  uint64_t made_round = 0;     // proposal rounds drawn (Philox counter)
  float2* chain_lp = nullptr;  // cached log psi of the chains
  float* chain_lq = nullptr;   // cached log q of the chains
  int8_t* prop = nullptr;      // proposals [C][N]
  float* prop_lq = nullptr;
  float2* prop_lp = nullptr;
  bool chain_cache = false;
  // autoregressive ansatz: FP64 master parameters (the FP32 copy is `made`)
  double* ar_params = nullptr;
  int64_t ar_P = 0;
  // CNN-ELU ansatz: FP64 master [alpha(N+1)], FP32 copies, its own Metropolis counter
  double* cnn_params = nullptr;
  float *cnn_W = nullptr, *cnn_b = nullptr;
  int64_t cnn_P = 0;
  uint64_t cnn_sweep = 0;
  bool cnn_thermalized = false;
};

}  // namespace

struct vmc_ctx {
  vmc_config cfg;
  cudaStream_t st = nullptr;
  std::vector<LatticeState> lats;
  int64_t Ns = 0;
  int Nmax = 0, Mmax = 0;
  int64_t Pmax = 0;
  bool dense = false;
  // per-step workspaces (sized for the largest lattice)
  int8_t* s_spins = nullptr;      // [Ns][Nmax]
  float2* s_T = nullptr;          // [Ns][Mmax]
  float2* s_E = nullptr;          // [Ns]
  double* estats = nullptr;       // [4]
  double* partial = nullptr;      // moments scratch
  double2* meanO = nullptr;       // [Pmax]
  float4* mean2 = nullptr;        // [Pmax] <O> as FP32 hi/lo pairs
  double2* F = nullptr;           // [Pmax]
  double2* x = nullptr;           // [Pmax]
  int64_t rows_pad = 0, ld = 0;
  float* X32 = nullptr;
  __nv_bfloat16* Xhi = nullptr;
  __nv_bfloat16* Xlo = nullptr;
  double2* S = nullptr;           // [Pmax][Pmax]
  float2* gpart = nullptr;        // split-K partials of the Gram (small P)
  int64_t gpart_cap = 0;
  SolveWork sw{};
  CgWork cg{};
  MadeWork mw{};
  int64_t made_cap = 0;           // rows of the MADE batch workspaces
  TdvpWork tw{};                  // TDVP workspaces (cfg.tdvp)
  // autoregressive ansatz (cfg.ar_ansatz)
  int8_t* ar_conn = nullptr;      // [Ns][Kmax][Nmax] connected configurations
  float* ar_lqc = nullptr;        // [Ns][Kmax] their log q
  float* ar_lq = nullptr;         // [Ns] log q of the samples
  double* ar_part = nullptr;      // moments chunk partials
  int64_t ar_part_cap = 0;
  int ar_Kmax = 0;
  float* cnn_O = nullptr;         // [Ns][P] dense log-derivatives of the CNN ansatz
  // batched sampler
  SampleArgs* d_bargs = nullptr;  // [n_lattices] device descriptors
  int* d_order = nullptr;         // heavy-first lattice order
  int* d_ustart = nullptr;        // first work unit of each lattice in that order (+ total)
  unsigned* d_counter = nullptr;  // work-queue counter
  int8_t* chain_backup = nullptr; // chains of all lattices (autotuning runs restore them)
  int tuned_wpb = 0, tuned_grid = 0, tuned_mpl = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t cap_st = nullptr;  // private stream the graph is captured on (the context's
                                  // own stream may be the legacy default stream)
  int g_therm = -1, g_samples = -1;  // arguments the captured graph was made for
  std::vector<uint64_t> g_sweep;      // sweep counters the device descriptors hold
  int8_t* g_spins = nullptr;
  float* g_eloc = nullptr;
  unsigned* status = nullptr;
  unsigned long long* n_accept = nullptr;
  int64_t launches = 0;
  int64_t psd_retries = 0;        // SR steps whose S was re-formed with the fourth product
  std::vector<void*> allocs;
  cudaEvent_t ev[8] = {};
  std::string err;
};

namespace {

vmc_status fail(vmc_ctx* c, vmc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

vmc_status cuda_fail(vmc_ctx* c, cudaError_t e, const char* where) {
  return fail(c, VMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
  } while (0)

template <typename T>
cudaError_t dalloc(vmc_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T));
  if (e != cudaSuccess) return e;
  ctx->allocs.push_back(v);
  *p = static_cast<T*>(v);
  return cudaSuccess;
}

int moves_of(const LatticeState& L);
RbmDev rbm_of(const LatticeState& L) {
  return RbmDev{L.N, L.M, L.a, L.b, L.Wt, L.mth, L.mlc, L.mlc + moves_of(L)};
}

int moves_of(const LatticeState& L) { return L.lat.model == 1 ? L.nb : L.N; }

LatDev lat_of(const LatticeState& L) {
  return LatDev{L.lat.model, L.lat.Lx, L.lat.Ly, L.nb, (float)L.lat.J, (float)L.lat.h};
}

// read and clear the device status word (synchronises)
vmc_status check_status(vmc_ctx* ctx, const char* where) {
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, where);
  if (h) {
    cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), ctx->st);
    if (h & DEV_ERR_TIMEOUT) return fail(ctx, VMC_ERR_TIMEOUT, std::string(where) + ": device wait expired");
    if (h & DEV_ERR_BOUNDS) return fail(ctx, VMC_ERR_ARG, std::string(where) + ": device index check failed");
    return fail(ctx, VMC_ERR_NUMERIC, std::string(where) + ": non-finite value or non-positive pivot");
  }
  return VMC_OK;
}

MadeDev made_of(vmc_ctx* ctx, LatticeState& L) {
  return made_view(L.made, L.W1t, L.W2t, L.W3t, L.N, ctx->cfg.made_hidden);
}

vmc_status lattice_ok(vmc_ctx* ctx, int lattice) {
  if (!ctx) return VMC_ERR_ARG;
  if (lattice < 0 || lattice >= (int)ctx->lats.size())
    return fail(ctx, VMC_ERR_ARG, "lattice index out of range");
  return VMC_OK;
}

vmc_status refresh_fp32(vmc_ctx* ctx, LatticeState& L) {
  CK(launch_param_prep(L.params, L.N, L.M, L.a, L.b, L.Wt, ctx->st), "param_prep");
  CK(launch_move_tables(L.params, L.N, L.M, L.lat.model, L.lat.Lx, L.lat.Ly, L.mth, L.mlc,
                        L.mlc + moves_of(L),
                        ctx->st), "move_tables");
  ++ctx->launches;
  ++ctx->launches;
  return VMC_OK;
}

// S of a sample set with T = tanh theta already in ctx->s_T; E may be null.  S_out (FP64)
// may be null when `fused` (tensor-core Gram only, the SR step): the Gram then writes the
// shifted lower triangle that the preconditioner's factorisation takes (ctx->sw.A32)
// directly.
vmc_status qfm_core(vmc_ctx* ctx, LatticeState& L, const int8_t* spins, const float2* E,
                    int64_t n, int precision, double2* S_out, bool mirror, bool fused = false,
                    bool lolo = false) {
  CK(launch_moments(spins, ctx->s_T, E, ctx->estats, n, L.N, L.M, ctx->partial, ctx->meanO,
                    E ? ctx->F : nullptr, ctx->st), "moments");
  ctx->launches += 2;
  const int64_t rows = 2 * L.P;
  const int64_t rows_pad = (rows + 127) / 128 * 128;
  const int64_t ld = (n + 63) / 64 * 64;
  if (rows_pad > ctx->rows_pad || ld > ctx->ld) return fail(ctx, VMC_ERR_ARG, "S workspace too small");
  const double inv_n = 1.0 / (double)n;
  if (precision == VMC_PREC_BF16SPLIT) {
    // In the SR step (fused) S only feeds the factor that preconditions CG on the exact
    // operator: one FP16 product (an 11-bit mantissa), no FP32 pair copy of S.  Elsewhere,
    // and when a factorisation met a non-positive pivot (lolo), the BF16 hi/lo split.
    const int prod = lolo ? 4 : fused ? 1 : 3;
    __half* x16 = prod == 1 ? reinterpret_cast<__half*>(ctx->Xhi) : nullptr;
    CK(launch_build_x(spins, ctx->s_T, ctx->meanO, ctx->mean2, n, L.N, L.M, rows_pad, ld, nullptr,
                      prod == 1 ? nullptr : ctx->Xhi, prod == 1 ? nullptr : ctx->Xlo, x16,
                      ctx->st), "build_x");
    ctx->launches += 2;
    cudaEventRecord(ctx->ev[6], ctx->st);
    cudaError_t e = launch_gram_tc(ctx->Xhi, ctx->Xlo, rows_pad, ld, L.P, inv_n, S_out, mirror,
                                   nullptr, fused ? ctx->sw.A32 : nullptr,
                                   ctx->cfg.shift, ctx->cfg.shift_mode, prod, ctx->gpart,
                                   ctx->gpart_cap, ctx->status, ctx->st);
    cudaEventRecord(ctx->ev[7], ctx->st);
    if (e == cudaErrorNotSupported) return fail(ctx, VMC_ERR_ARG, "tensor-core Gram: shape not supported");
    CK(e, "gram_tc");
    ++ctx->launches;
  } else {
    CK(launch_build_x(spins, ctx->s_T, ctx->meanO, ctx->mean2, n, L.N, L.M, rows_pad, ld, ctx->X32, nullptr,
                      nullptr, nullptr, ctx->st), "build_x");
    ctx->launches += 2;
    cudaEventRecord(ctx->ev[6], ctx->st);
    CK(launch_gram_f32(ctx->X32, rows_pad, ld, L.P, inv_n, S_out, mirror, ctx->gpart,
                       ctx->gpart_cap, ctx->st), "gram_f32");
    cudaEventRecord(ctx->ev[7], ctx->st);
    ++ctx->launches;
  }
  return VMC_OK;
}

// S (FP64) may be null for the mixed solvers when the Gram already wrote their inputs.
vmc_status solve_core(vmc_ctx* ctx, int64_t P, const double2* S, const double2* F,
                      double2* x, int* iters, double* relres) {
  ctx->sw.P = P;
  const vmc_config& c = ctx->cfg;
  int it = 0;
  double rel = 0.0;
  if (c.solver == VMC_SOLVER_CHOLESKY_FP64) {
    CK(solve_cholesky_fp64(S, F, x, c.shift, c.shift_mode, ctx->sw, ctx->status, ctx->st,
                           &ctx->launches), "cholesky_fp64");
    CK(residual_fp64(S, F, x, c.shift, c.shift_mode, ctx->sw, ctx->st, &rel), "residual");
    ctx->launches += 2;
  } else if (c.solver == VMC_SOLVER_CHOLESKY_MIXED || c.solver == VMC_SOLVER_CHOLESKY_TC) {
    if (S) {
      CK(split_shift(S, c.shift, c.shift_mode, ctx->sw, ctx->st), "split_shift");
      ++ctx->launches;
    }
    CK(solve_cholesky_mixed(F, x, c.shift, c.shift_mode, c.cg_tol, c.cg_maxit,
                            c.solver == VMC_SOLVER_CHOLESKY_TC, ctx->sw, ctx->status, ctx->st,
                            &ctx->launches, &it, &rel), "cholesky_mixed");
  } else {
    return fail(ctx, VMC_ERR_ARG, "solver not available for a dense S");
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  vmc_status s = check_status(ctx, "solve");
  if (s != VMC_OK) return s;
  if (!(rel == rel) || (c.solver != VMC_SOLVER_CHOLESKY_FP64 && !(rel <= c.cg_tol)))
    return fail(ctx, VMC_ERR_NUMERIC, "iterative refinement did not reach the tolerance");
  return VMC_OK;
}

}  // namespace

extern "C" {

vmc_status vmc_init(const vmc_config* cfg, const vmc_lattice* lattices, int n_lattices,
                    void* stream, vmc_ctx** out) {
  if (!cfg || !lattices || !out || n_lattices < 1 || n_lattices > 4096) return VMC_ERR_ARG;
  *out = nullptr;
  if (cfg->n_chains < 1 || cfg->samples_per_chain < 1 || cfg->sweeps_per_sample < 1 ||
      cfg->therm_sweeps < 0 || cfg->sweep_len < 0)
    return VMC_ERR_ARG;
  if (cfg->precision != VMC_PREC_FP32 && cfg->precision != VMC_PREC_BF16SPLIT) return VMC_ERR_ARG;
  if (cfg->solver < 0 || cfg->solver > 3 || (cfg->shift_mode != 0 && cfg->shift_mode != 1))
    return VMC_ERR_ARG;
  if (!(cfg->shift >= 0.0)) return VMC_ERR_ARG;
  if (cfg->made_hidden < 0 || cfg->made_hidden > 512 || cfg->made_hidden % 32 != 0 ||
      cfg->made_batch < 0 || (cfg->tdvp != 0 && cfg->tdvp != 1) ||
      (cfg->ar_ansatz != 0 && cfg->ar_ansatz != 1))
    return VMC_ERR_ARG;
  if (cfg->ar_ansatz && (cfg->made_hidden <= 0 || cfg->solver == VMC_SOLVER_CG)) return VMC_ERR_ARG;
  if ((cfg->cnn_ansatz != 0 && cfg->cnn_ansatz != 1) || (cfg->cnn_ansatz && !cfg->tdvp)) return VMC_ERR_ARG;
  for (int l = 0; l < n_lattices; ++l) {
    const vmc_lattice& L = lattices[l];
    const int N = L.Lx * L.Ly;
    if ((L.model != 0 && L.model != 1) || L.Lx < 1 || L.Ly < 1 || N < 2 || N > 1024 ||
        L.alpha < 1 || L.alpha * N > 512)
      return VMC_ERR_ARG;
  }
  vmc_ctx* ctx = new vmc_ctx();
  ctx->cfg = *cfg;
  ctx->st = static_cast<cudaStream_t>(stream);
  ctx->Ns = (int64_t)cfg->n_chains * cfg->samples_per_chain;
  for (int l = 0; l < n_lattices; ++l) {
    LatticeState S;
    S.lat = lattices[l];
    S.N = S.lat.Lx * S.lat.Ly;
    S.M = S.lat.alpha * S.N;
    S.nb = num_bonds(S.lat.Lx, S.lat.Ly);
    S.P = (int64_t)S.N + S.M + (int64_t)S.N * S.M;
    ctx->Nmax = std::max(ctx->Nmax, S.N);
    ctx->Mmax = std::max(ctx->Mmax, S.M);
    ctx->Pmax = std::max(ctx->Pmax, S.P);
    if (cfg->cnn_ansatz) {
      if (S.lat.Ly != 1 || S.lat.model != 0 || S.lat.alpha * S.N > 512) {
        delete ctx;
        return VMC_ERR_ARG;
      }
      S.cnn_P = (int64_t)S.lat.alpha * (S.N + 1);
      ctx->Pmax = std::max(ctx->Pmax, S.cnn_P);
    }
    if (cfg->ar_ansatz) {
      S.ar_P = made_nparams(S.N, cfg->made_hidden);
      ctx->Pmax = std::max(ctx->Pmax, S.ar_P);
      ctx->ar_Kmax = std::max(ctx->ar_Kmax, S.lat.model == 0 ? S.N : num_bonds(S.lat.Lx, S.lat.Ly));
    }
    ctx->lats.push_back(S);
  }
  for (auto& L : ctx->lats)
    if (cfg->ar_ansatz && L.ar_P > 16384) {
      delete ctx;
      return VMC_ERR_ARG;
    }
  ctx->dense = cfg->solver != VMC_SOLVER_CG;
  auto oom = [&](cudaError_t e) {
    vmc_destroy(ctx);
    (void)e;
    cudaGetLastError();
    return VMC_ERR_OOM;
  };
  cudaError_t e;
  for (auto& L : ctx->lats) {
    if ((e = dalloc(ctx, &L.params, L.P)) || (e = dalloc(ctx, &L.a, L.N)) ||
        (e = dalloc(ctx, &L.b, L.M)) || (e = dalloc(ctx, &L.Wt, (size_t)L.N * L.M)) ||
        (e = dalloc(ctx, &L.mth, (size_t)moves_of(L) * L.M)) ||
        (e = dalloc(ctx, &L.mlc, (size_t)3 * moves_of(L))) ||   // mlc [moves], mpre [moves][2]
        (e = dalloc(ctx, &L.chains, (size_t)cfg->n_chains * L.N)))
      return oom(e);
    cudaMemset(L.params, 0, L.P * sizeof(double2));
    std::vector<int8_t> up((size_t)cfg->n_chains * L.N, 1);
    cudaMemcpy(L.chains, up.data(), up.size(), cudaMemcpyHostToDevice);
    launch_param_prep(L.params, L.N, L.M, L.a, L.b, L.Wt, ctx->st);
    launch_move_tables(L.params, L.N, L.M, L.lat.model, L.lat.Lx, L.lat.Ly, L.mth, L.mlc,
                       L.mlc + moves_of(L), ctx->st);
    if (cfg->made_hidden > 0) {
      const int H = cfg->made_hidden;
      const int64_t np = made_nparams(L.N, H);
      const size_t C = (size_t)cfg->n_chains;
      if ((e = dalloc(ctx, &L.made, np)) || (e = dalloc(ctx, &L.made_m, np)) ||
          (e = dalloc(ctx, &L.made_v, np)) || (e = dalloc(ctx, &L.made_g, np)) ||
          (e = dalloc(ctx, &L.W1t, (size_t)H * L.N)) || (e = dalloc(ctx, &L.W2t, (size_t)H * H)) ||
          (e = dalloc(ctx, &L.W3t, (size_t)H * L.N)) || (e = dalloc(ctx, &L.chain_lp, C)) ||
          (e = dalloc(ctx, &L.chain_lq, C)) || (e = dalloc(ctx, &L.prop, C * L.N)) ||
          (e = dalloc(ctx, &L.prop_lq, C)) || (e = dalloc(ctx, &L.prop_lp, C)))
        return oom(e);
      cudaMemset(L.made, 0, np * sizeof(float));
      cudaMemset(L.made_m, 0, np * sizeof(float));
      cudaMemset(L.made_v, 0, np * sizeof(float));
      launch_made_transpose(made_view(L.made, L.W1t, L.W2t, L.W3t, L.N, H), ctx->st);
      if (cfg->ar_ansatz) {
        if ((e = dalloc(ctx, &L.ar_params, np))) return oom(e);
        cudaMemset(L.ar_params, 0, np * sizeof(double));
      }
    }
    if (cfg->cnn_ansatz) {
      if ((e = dalloc(ctx, &L.cnn_params, L.cnn_P)) ||
          (e = dalloc(ctx, &L.cnn_W, (size_t)L.lat.alpha * L.N)) ||
          (e = dalloc(ctx, &L.cnn_b, (size_t)L.lat.alpha)))
        return oom(e);
      cudaMemset(L.cnn_params, 0, L.cnn_P * sizeof(double));
      launch_cnn_prep(L.cnn_params, L.lat.alpha, L.N, L.cnn_W, L.cnn_b, ctx->st);
    }
  }
  {
    size_t chain_bytes = 0;
    for (auto& L : ctx->lats) chain_bytes += (size_t)cfg->n_chains * L.N;
    if ((e = dalloc(ctx, &ctx->d_bargs, ctx->lats.size())) ||
        (e = dalloc(ctx, &ctx->d_order, ctx->lats.size())) ||
        (e = dalloc(ctx, &ctx->d_ustart, ctx->lats.size() + 1)) || (e = dalloc(ctx, &ctx->d_counter, 1)) ||
        (e = dalloc(ctx, &ctx->chain_backup, chain_bytes)))
      return oom(e);
  }
  if (cfg->made_hidden > 0) {
    const int H = cfg->made_hidden;
    int64_t B = std::max<int64_t>(cfg->made_batch > 0 ? cfg->made_batch : 4096, cfg->n_chains);
    if (cfg->ar_ansatz) B = std::max<int64_t>(B, (int64_t)cfg->n_chains * cfg->samples_per_chain);
    ctx->made_cap = B;
    if ((e = dalloc(ctx, &ctx->mw.logq, B)) || (e = dalloc(ctx, &ctx->mw.H1, (size_t)B * H)) ||
        (e = dalloc(ctx, &ctx->mw.H2, (size_t)B * H)) || (e = dalloc(ctx, &ctx->mw.G1, (size_t)B * H)) ||
        (e = dalloc(ctx, &ctx->mw.G2, (size_t)B * H)) ||
        (e = dalloc(ctx, &ctx->mw.G3, (size_t)B * ctx->Nmax)))
      return oom(e);
  }
  const int64_t Ns = ctx->Ns;
  if ((e = dalloc(ctx, &ctx->s_spins, (size_t)Ns * ctx->Nmax)) ||
      (e = dalloc(ctx, &ctx->s_T, (size_t)Ns * ctx->Mmax)) || (e = dalloc(ctx, &ctx->s_E, (Ns + 255) / 256 * 256)) ||
      (e = dalloc(ctx, &ctx->estats, 8)) ||
      (e = dalloc(ctx, &ctx->partial, (size_t)moments_partial_doubles(Ns, ctx->Nmax, ctx->Mmax))) ||
      (e = dalloc(ctx, &ctx->meanO, ctx->Pmax)) || (e = dalloc(ctx, &ctx->mean2, ctx->Pmax)) || (e = dalloc(ctx, &ctx->F, ctx->Pmax)) ||
      (e = dalloc(ctx, &ctx->x, ctx->Pmax)) || (e = dalloc(ctx, &ctx->status, 1)) ||
      (e = dalloc(ctx, &ctx->n_accept, 1)))
    return oom(e);
  {
    CgWork& w = ctx->cg;
    const int64_t P = ctx->Pmax;
    if ((e = dalloc(ctx, &w.r, P)) || (e = dalloc(ctx, &w.p, P)) || (e = dalloc(ctx, &w.q, P)) ||
        (e = dalloc(ctx, &w.y, P)) || (e = dalloc(ctx, &w.z, P)) ||
        (e = dalloc(ctx, &w.D, P)) ||
        (e = dalloc(ctx, &w.Minv, P)) || (e = dalloc(ctx, &w.t2, ctx->Mmax)) ||
        (e = dalloc(ctx, &w.t2part, (size_t)CG_T2_BLOCKS * ctx->Mmax)) ||
        (e = dalloc(ctx, &w.va, ctx->Nmax)) || (e = dalloc(ctx, &w.vb, ctx->Mmax + 128)) ||
        (e = dalloc(ctx, &w.V, (size_t)ctx->Nmax * ctx->Mmax)) || (e = dalloc(ctx, &w.u, (Ns + 255) / 256 * 256)) ||
        (e = dalloc(ctx, &w.upart, (size_t)cg_partial_floats2(Ns, ctx->Mmax))) ||
        (e = dalloc(ctx, &w.ustats, 8)) || (e = dalloc(ctx, &w.vpart, CG_VPART_DOUBLES)) ||
        (e = dalloc(ctx, &w.sc, 8)) || (e = dalloc(ctx, &w.flag, 8)) ||
        (e = dalloc(ctx, &w.ones, (Ns + 255) / 256 * 256)) || (e = dalloc(ctx, &w.zero2, 2)))
      return oom(e);
    w.mpart = ctx->partial;
    // u and E stay finite beyond the sample count (the O^H u kernel reads whole 64-sample
    // blocks); the flags' upper half, the zero mean and the ones are constants
    const size_t npad = (size_t)((Ns + 255) / 256 * 256);
    if ((e = cudaMemset(w.u, 0, sizeof(float2) * npad)) != cudaSuccess ||
        (e = cudaMemset(ctx->s_E, 0, sizeof(float2) * npad)) != cudaSuccess ||
        (e = cudaMemset(w.flag, 0, 8 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(w.zero2, 0, 2 * sizeof(double))) != cudaSuccess ||
        (e = fill_ones(w.ones, (int64_t)npad)) != cudaSuccess)
      return oom(e);
    if (!ctx->dense && cfg->precision == VMC_PREC_BF16SPLIT) {
      // operator products on the tensor cores: operand planes sized for the largest lattice
      // (every lattice's shape is bounded by the largest N, M; the OhU grid by the SMs)
      const CgTcShape sh = cg_tc_shape(ctx->Nmax, ctx->Mmax, Ns);
      const int64_t sms = persistent_grid(1 << 20);
      w.cap_sb = sh.s_rows * sh.kN;
      w.cap_bs = sh.b_rows * sh.ldK;
      w.cap_v = sh.v_rows * sh.kN;
      w.cap_part2 = sms * 128 * 256;
      w.cap_yb = sms * ctx->Mmax;
      w.cap_ov = sms;
      if ((e = dalloc(ctx, &w.Sb, (size_t)w.cap_sb)) || (e = dalloc(ctx, &w.Bs, (size_t)w.cap_bs)) ||
          (e = dalloc(ctx, &w.Vhi, (size_t)w.cap_v)) || (e = dalloc(ctx, &w.Vlo, (size_t)w.cap_v)) ||
          (e = dalloc(ctx, &w.part2, (size_t)w.cap_part2)) ||
          (e = dalloc(ctx, &w.ybpart, (size_t)w.cap_yb)) ||
          (e = dalloc(ctx, &w.ovpart, (size_t)w.cap_ov)))
        return oom(e);
    }
  }
  if (cfg->cnn_ansatz) {
    int64_t pc = 0;
    for (auto& L : ctx->lats) pc = std::max(pc, L.cnn_P);
    if ((e = dalloc(ctx, &ctx->cnn_O, (size_t)Ns * pc))) return oom(e);
  }
  if (cfg->ar_ansatz) {
    const size_t K = (size_t)ctx->ar_Kmax;
    ctx->ar_part_cap = 2 * ctx->Pmax * 512;
    if ((e = dalloc(ctx, &ctx->ar_conn, (size_t)Ns * K * ctx->Nmax)) ||
        (e = dalloc(ctx, &ctx->ar_lqc, (size_t)Ns * K)) || (e = dalloc(ctx, &ctx->ar_lq, (size_t)Ns)) ||
        (e = dalloc(ctx, &ctx->ar_part, (size_t)ctx->ar_part_cap)))
      return oom(e);
  }
  if (cfg->tdvp) {
    // TDVP workspaces: FP64 S, Q, the Jacobi work matrix, V and the integrator's S at y
    TdvpWork& tw = ctx->tw;
    const int64_t P = ctx->Pmax;
    if (P > 4096) {
      vmc_destroy(ctx);
      return VMC_ERR_ARG;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    tw.n_sm = sms;
    tw.Pcap = P;
    tw.ncap = Ns;
    tw.status = ctx->status;
    tw.red_cap = 64 * sms;
    tw.mom_part_cap = 2 * P * 512;
    tw.gram_part_cap = tdvp_gram_partial_doubles2(Ns, P, sms);
    if ((e = dalloc(ctx, &tw.w, (size_t)Ns)) || (e = dalloc(ctx, &tw.lp, (size_t)Ns)) ||
        (e = dalloc(ctx, &tw.estats, 8)) || (e = dalloc(ctx, &tw.meanO, P)) ||
        (e = dalloc(ctx, &tw.F, P)) || (e = dalloc(ctx, &tw.mom_part, (size_t)tw.mom_part_cap)) ||
        (e = dalloc(ctx, &tw.gram_part, (size_t)tw.gram_part_cap)) ||
        (e = dalloc(ctx, &tw.S, (size_t)P * P)) || (e = dalloc(ctx, &tw.Q, (size_t)P * P)) ||
        (e = dalloc(ctx, &tw.A, (size_t)P * P)) || (e = dalloc(ctx, &tw.V, (size_t)P * P)) ||
        (e = dalloc(ctx, &tw.S0, (size_t)P * P)) || (e = dalloc(ctx, &tw.lam, P)) ||
        (e = dalloc(ctx, &tw.rot, P + 2)) || (e = dalloc(ctx, &tw.bar, 4)) ||
        (e = dalloc(ctx, &tw.red, (size_t)tw.red_cap)) || (e = dalloc(ctx, &tw.info, 2)) ||
        (e = dalloc(ctx, &tw.rho, P)) || (e = dalloc(ctx, &tw.qd, P)) ||
        (e = dalloc(ctx, &tw.lamp, P)) || (e = dalloc(ctx, &tw.lstats, 4)) ||
        (e = dalloc(ctx, &tw.qpart, (size_t)(P + 255) / 256 + 1)))
      return oom(e);
    for (int k = 0; k < 8; ++k)
      if ((e = dalloc(ctx, &tw.vec[k], P))) return oom(e);
    if ((e = dalloc(ctx, &tw.lp2, (size_t)Ns)) || (e = dalloc(ctx, &tw.e2, (size_t)Ns)) ||
        (e = dalloc(ctx, &tw.osc, (size_t)Ns)) || (e = dalloc(ctx, &tw.eexc, (size_t)Ns)) ||
        (e = dalloc(ctx, &tw.wraw, (size_t)Ns)) || (e = dalloc(ctx, &tw.olap, 8)))
      return oom(e);
  }
  if (ctx->dense) {
    const int64_t P = ctx->Pmax;
    ctx->rows_pad = (2 * P + 127) / 128 * 128;
    ctx->ld = (Ns + 63) / 64 * 64;
    const size_t xs = (size_t)ctx->rows_pad * ctx->ld;
    const int64_t nblk = (P + 63) / 64;
    if ((e = dalloc(ctx, &ctx->X32, xs)) || (e = dalloc(ctx, &ctx->Xhi, xs)) ||
        (e = dalloc(ctx, &ctx->Xlo, xs)) || (e = dalloc(ctx, &ctx->S, (size_t)P * P)) ||
        (e = dalloc(ctx, &ctx->sw.r, P)) || (e = dalloc(ctx, &ctx->sw.c, P)) ||
        (e = dalloc(ctx, &ctx->sw.r32, P)) || (e = dalloc(ctx, &ctx->sw.y32, P)) ||
        (e = dalloc(ctx, &ctx->sw.c32, P)) || (e = dalloc(ctx, &ctx->sw.scal, 8)) ||
        (e = dalloc(ctx, &ctx->sw.scal_part, 256)) ||
        (e = dalloc(ctx, &ctx->sw.bar, 128)) ||
        (e = dalloc(ctx, &ctx->sw.fin, P)))
      return oom(e);
    // split-K Gram partials: up to 8M complex FP32 (64 MB), used only when P is small
    ctx->gpart_cap = std::min<int64_t>((int64_t)1 << 23, P * P * 64);
    if ((e = dalloc(ctx, &ctx->gpart, (size_t)ctx->gpart_cap))) return oom(e);
    ctx->sw.Xhi = ctx->Xhi;
    ctx->sw.Xlo = ctx->Xlo;
    ctx->sw.x_elems = (int64_t)xs;
    const size_t nsb = (size_t)((P + 255) / 256);
    if (cfg->solver == VMC_SOLVER_CHOLESKY_FP64) {
      if ((e = dalloc(ctx, &ctx->sw.A64, (size_t)P * P)) ||
          (e = dalloc(ctx, &ctx->sw.D64, (size_t)nblk * 64 * 64)) ||
          (e = dalloc(ctx, &ctx->sw.T64f, nsb * 256 * 256)) ||
          (e = dalloc(ctx, &ctx->sw.T64b, nsb * 256 * 256)))
        return oom(e);
    } else {
      if ((e = dalloc(ctx, &ctx->sw.A32, (size_t)P * P)) ||
          (e = dalloc(ctx, &ctx->sw.D32, (size_t)nblk * 64 * 64)) ||
          (e = dalloc(ctx, &ctx->sw.T32f, nsb * 256 * 256)) ||
          (e = dalloc(ctx, &ctx->sw.T32b, nsb * 256 * 256)) ||
          (e = dalloc(ctx, &ctx->sw.S2, (size_t)P * P)) || (e = dalloc(ctx, &ctx->sw.x2, P)) ||
          (e = dalloc(ctx, &ctx->sw.dsc, P)))
        return oom(e);
    }
  }
  cudaMemset(ctx->status, 0, sizeof(unsigned));
  for (auto& ev : ctx->ev) cudaEventCreate(&ev);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    vmc_destroy(ctx);
    return VMC_ERR_CUDA;
  }
  ctx->launches = (int64_t)ctx->lats.size();
  *out = ctx;
  return VMC_OK;
}

void vmc_destroy(vmc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
  for (void* p : ctx->allocs) cudaFree(p);
  for (auto& ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  delete ctx;
}

const char* vmc_last_error(const vmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t vmc_kernel_launches(const vmc_ctx* ctx) { return ctx ? ctx->launches : 0; }
int64_t vmc_num_samples(const vmc_ctx* ctx) { return ctx ? ctx->Ns : 0; }
int64_t vmc_num_params(const vmc_ctx* ctx, int lattice) {
  if (!ctx || lattice < 0 || lattice >= (int)ctx->lats.size()) return 0;
  return ctx->lats[lattice].P;
}

vmc_status vmc_set_params(vmc_ctx* ctx, int lattice, const double* params_host) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (!params_host) return fail(ctx, VMC_ERR_ARG, "params_host is NULL");
  LatticeState& L = ctx->lats[lattice];
  CK(cudaMemcpyAsync(L.params, params_host, L.P * sizeof(double2), cudaMemcpyHostToDevice, ctx->st),
     "set_params");
  if ((s = refresh_fp32(ctx, L))) return s;
  CK(cudaStreamSynchronize(ctx->st), "set_params");
  L.chain_cache = false;
  return VMC_OK;
}

vmc_status vmc_get_params(vmc_ctx* ctx, int lattice, double* params_host) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (!params_host) return fail(ctx, VMC_ERR_ARG, "params_host is NULL");
  LatticeState& L = ctx->lats[lattice];
  CK(cudaMemcpyAsync(params_host, L.params, L.P * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st),
     "get_params");
  CK(cudaStreamSynchronize(ctx->st), "get_params");
  return VMC_OK;
}

vmc_status vmc_set_chains(vmc_ctx* ctx, int lattice, const int8_t* spins_host) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (!spins_host) return fail(ctx, VMC_ERR_ARG, "spins_host is NULL");
  LatticeState& L = ctx->lats[lattice];
  const size_t bytes = (size_t)ctx->cfg.n_chains * L.N;
  for (size_t k = 0; k < bytes; ++k)
    if (spins_host[k] != 1 && spins_host[k] != -1) return fail(ctx, VMC_ERR_ARG, "spins must be +1 or -1");
  CK(cudaMemcpyAsync(L.chains, spins_host, bytes, cudaMemcpyHostToDevice, ctx->st), "set_chains");
  CK(cudaStreamSynchronize(ctx->st), "set_chains");
  L.sweep = 0;
  L.thermalized = false;
  L.chain_cache = false;
  return VMC_OK;
}

vmc_status vmc_get_chains(vmc_ctx* ctx, int lattice, int8_t* spins_host) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (!spins_host) return fail(ctx, VMC_ERR_ARG, "spins_host is NULL");
  LatticeState& L = ctx->lats[lattice];
  CK(cudaMemcpyAsync(spins_host, L.chains, (size_t)ctx->cfg.n_chains * L.N, cudaMemcpyDeviceToHost,
                     ctx->st), "get_chains");
  CK(cudaStreamSynchronize(ctx->st), "get_chains");
  return VMC_OK;
}

// theta of n configurations with the context's precision (the chains' starting cache)
static cudaError_t theta_of(vmc_ctx* ctx, LatticeState& L, const int8_t* spins, int64_t n,
                            float2* theta) {
  if (ctx->cfg.precision == VMC_PREC_BF16SPLIT)
    return launch_theta_tc(rbm_of(L), spins, n, theta, ctx->status, ctx->st);
  return launch_theta_gemm(rbm_of(L), spins, n, theta, ctx->st);
}

vmc_status vmc_theta(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* theta) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && (!spins || !theta))) return fail(ctx, VMC_ERR_ARG, "bad batch");
  if (n == 0) return VMC_OK;
  LatticeState& L = ctx->lats[lattice];
  CK(theta_of(ctx, L, spins, n, reinterpret_cast<float2*>(theta)), "theta");
  ++ctx->launches;
  return check_status(ctx, "theta");
}

vmc_status vmc_logpsi(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* logpsi) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && (!spins || !logpsi))) return fail(ctx, VMC_ERR_ARG, "bad batch");
  if (n == 0) return VMC_OK;
  LatticeState& L = ctx->lats[lattice];
  CK(launch_logpsi(rbm_of(L), spins, n, reinterpret_cast<float2*>(logpsi), ctx->status, ctx->st),
     "logpsi");
  ++ctx->launches;
  return VMC_OK;
}

vmc_status vmc_local_energy(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                            float* eloc) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && (!spins || !eloc))) return fail(ctx, VMC_ERR_ARG, "bad batch");
  if (n == 0) return VMC_OK;
  LatticeState& L = ctx->lats[lattice];
  CK(launch_eloc(rbm_of(L), lat_of(L), spins, n, reinterpret_cast<float2*>(eloc), ctx->status,
                 ctx->st), "local_energy");
  ++ctx->launches;
  return VMC_OK;
}

vmc_status vmc_sample(vmc_ctx* ctx, int lattice, int n_therm, int n_samples, int8_t* spins_out,
                      float* logpsi_out, float* eloc_out) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (n_therm < 0 || n_samples < 0) return fail(ctx, VMC_ERR_ARG, "negative sweep count");
  LatticeState& L = ctx->lats[lattice];
  SampleArgs A{};
  A.rbm = rbm_of(L);
  A.lat = lat_of(L);
  A.chains = L.chains;
  A.C = ctx->cfg.n_chains;
  A.L = ctx->cfg.sweep_len > 0 ? ctx->cfg.sweep_len : L.N;
  A.seed = ctx->cfg.seed;
  A.stream = (uint64_t)lattice;
  A.sweep0 = L.sweep;
  A.n_therm = n_therm;
  A.n_samples = n_samples;
  A.sweeps_per_sample = ctx->cfg.sweeps_per_sample;
  A.spins_out = spins_out;
  A.logpsi_out = reinterpret_cast<float2*>(logpsi_out);
  A.eloc_out = reinterpret_cast<float2*>(eloc_out);
  A.t_out = nullptr;
  A.n_accept = ctx->n_accept;
  A.status = ctx->status;
  if (n_therm + n_samples == 0) return VMC_OK;
  if (ctx->cfg.precision == VMC_PREC_BF16SPLIT) {
    // the chains start from the same theta as in vmc_sr_step (the t buffer is scratch here:
    // a chain reads its row before anything else is written there)
    CK(theta_of(ctx, L, L.chains, A.C, ctx->s_T), "theta");
    ++ctx->launches;
    A.theta_in = ctx->s_T;
  }
  CK(launch_sample(A, ctx->st), "sample");
  ++ctx->launches;
  L.sweep += (uint64_t)n_therm + (uint64_t)n_samples * ctx->cfg.sweeps_per_sample;
  if (n_therm > 0) L.thermalized = true;
  L.chain_cache = false;          // the chains moved: cached log psi / log q are stale
  return VMC_OK;
}

vmc_status vmc_grad(vmc_ctx* ctx, int lattice, const int8_t* spins, const float* eloc, int64_t n,
                    float* O_out, double* F_out, double* E_stats) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (n < 1 || n > ctx->Ns || !spins || !eloc) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  const float2* E = reinterpret_cast<const float2*>(eloc);
  CK(launch_theta_tanh(rbm_of(L), spins, n, ctx->s_T, ctx->st), "theta_tanh");
  CK(launch_estats(E, n, ctx->estats, ctx->status, ctx->st), "estats");
  CK(launch_moments(spins, ctx->s_T, E, ctx->estats, n, L.N, L.M, ctx->partial, ctx->meanO, ctx->F,
                    ctx->st), "moments");
  ctx->launches += 4;
  if (F_out)
    CK(cudaMemcpyAsync(F_out, ctx->F, L.P * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->st), "grad");
  if (O_out) {
    CK(launch_ok_dense(spins, ctx->s_T, n, L.N, L.M, reinterpret_cast<float2*>(O_out), ctx->st), "ok");
    ++ctx->launches;
  }
  if (E_stats) {
    CK(cudaMemcpyAsync(E_stats, ctx->estats, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st), "grad");
    return check_status(ctx, "grad");
  }
  return VMC_OK;
}

vmc_status vmc_qfm(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, int precision,
                   double* S_out) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (n < 1 || n > ctx->Ns || !spins || !S_out) return fail(ctx, VMC_ERR_ARG, "bad batch");
  if (!ctx->dense) return fail(ctx, VMC_ERR_STATE, "context was created for the CG solver (no dense S)");
  if (precision != VMC_PREC_FP32 && precision != VMC_PREC_BF16SPLIT) return fail(ctx, VMC_ERR_ARG, "bad precision");
  LatticeState& L = ctx->lats[lattice];
  CK(launch_theta_tanh(rbm_of(L), spins, n, ctx->s_T, ctx->st), "theta_tanh");
  ++ctx->launches;
  if ((s = qfm_core(ctx, L, spins, nullptr, n, precision, reinterpret_cast<double2*>(S_out), true)))
    return s;
  return check_status(ctx, "qfm");
}

vmc_status vmc_solve(vmc_ctx* ctx, int lattice, const double* S, const double* F, double* x,
                     int* iters, double* relres) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (!S || !F || !x) return fail(ctx, VMC_ERR_ARG, "NULL buffer");
  if (!ctx->dense) return fail(ctx, VMC_ERR_STATE, "context was created for the CG solver");
  LatticeState& L = ctx->lats[lattice];
  return solve_core(ctx, L.P, reinterpret_cast<const double2*>(S), reinterpret_cast<const double2*>(F),
                    reinterpret_cast<double2*>(x), iters, relres);
}

vmc_status vmc_cg_solve(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, const double* F,
                        double* x, int* iters, double* relres) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (n < 1 || n > ctx->Ns || !spins || !F || !x) return fail(ctx, VMC_ERR_ARG, "bad arguments");
  LatticeState& L = ctx->lats[lattice];
  const vmc_config& c = ctx->cfg;
  CK(launch_theta_tanh(rbm_of(L), spins, n, ctx->s_T, ctx->st), "theta_tanh");
  CK(launch_moments(spins, ctx->s_T, nullptr, ctx->estats, n, L.N, L.M, ctx->partial, ctx->meanO,
                    nullptr, ctx->st), "moments");
  ctx->launches += 3;
  CgProblem pb{spins, ctx->s_T, n, L.N, L.M, ctx->meanO,
               ctx->cg.Sb != nullptr && cg_tc_shape(L.N, L.M, n).ok, ctx->status};
  CK(cg_prepare(pb, ctx->cg, c.shift, c.shift_mode, ctx->st, &ctx->launches), "cg_prepare");
  int it = 0;
  double rel = 0.0;
  CK(cg_solve(pb, reinterpret_cast<const double2*>(F), reinterpret_cast<double2*>(x), c.cg_tol,
              c.cg_maxit, ctx->cg, ctx->st, &ctx->launches, &it, &rel), "cg_solve");
  if (iters) *iters = it;
  if (relres) *relres = rel;
  if ((s = check_status(ctx, "cg_solve"))) return s;
  if (!(rel == rel)) return fail(ctx, VMC_ERR_NUMERIC, "CG produced a non-finite residual");
  if (!(rel <= c.cg_tol))
    return fail(ctx, VMC_ERR_NUMERIC, "CG did not reach cg_tol within cg_maxit iterations "
                                      "(x holds the last iterate)");
  return VMC_OK;
}

vmc_status vmc_sr_apply(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                        const double* v, double* y) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (n < 1 || n > ctx->Ns || !spins || !v || !y) return fail(ctx, VMC_ERR_ARG, "bad arguments");
  if (ctx->dense) return fail(ctx, VMC_ERR_STATE, "context was created for a dense solver");
  LatticeState& L = ctx->lats[lattice];
  const vmc_config& c = ctx->cfg;
  CK(launch_theta_tanh(rbm_of(L), spins, n, ctx->s_T, ctx->st), "theta_tanh");
  CK(launch_moments(spins, ctx->s_T, nullptr, ctx->estats, n, L.N, L.M, ctx->partial, ctx->meanO,
                    nullptr, ctx->st), "moments");
  ctx->launches += 3;
  CgProblem pb{spins, ctx->s_T, n, L.N, L.M, ctx->meanO,
               ctx->cg.Sb != nullptr && cg_tc_shape(L.N, L.M, n).ok, ctx->status};
  CK(cg_prepare(pb, ctx->cg, c.shift, c.shift_mode, ctx->st, &ctx->launches), "cg_prepare");
  CK(cg_apply(pb, ctx->cg, reinterpret_cast<const double2*>(v), reinterpret_cast<double2*>(y),
              ctx->st, &ctx->launches), "cg_apply");
  CK(cudaStreamSynchronize(ctx->st), "cg_apply");
  return check_status(ctx, "cg_apply");
}

// The samples of one SR step (Ns = n_chains * samples_per_chain) from the lattice's chains:
// spins, E_loc and tanh(theta) into the step buffers; *steps = Metropolis steps per chain.
// The SR step's solve of S~ x = F.  With the BF16-split S (the tensor-core Gram writes the
// factor's input) the system solved is that of the samples' own S applied matrix-free in
// FP32 (the CG operator, O^H (O v) / n + D v), by conjugate gradients preconditioned with the
// Cholesky factor of the BF16-split S~: the split's rounding (about 2^-16 of |S_kl|) then
// only slows the iteration instead of moving the solution along the poorly conditioned
// directions of S~.  Otherwise solve_core on the formed S.  *rel_ex (may be null) receives
// the explicit residual of the preconditioned CG (the recursive one in *rel).
static vmc_status step_solve(vmc_ctx* ctx, LatticeState& L, bool fused, int* iters, double* rel,
                             double* rel_ex) {
  const vmc_config& c = ctx->cfg;
  if (!(fused && c.precision == VMC_PREC_BF16SPLIT)) {
    vmc_status s = solve_core(ctx, L.P, fused ? nullptr : ctx->S, ctx->F, ctx->x, iters, rel);
    if (rel_ex) *rel_ex = *rel;
    return s;
  }
  ctx->sw.P = L.P;
  CgProblem pb{ctx->s_spins, ctx->s_T, ctx->Ns, L.N, L.M, ctx->meanO, false, ctx->status};
  CK(cg_prepare(pb, ctx->cg, c.shift, c.shift_mode, ctx->st, &ctx->launches), "cg_prepare");
  CgWork& w = ctx->cg;
  PcgOperator apply = [&](const double2* v, double2* y) {
    return cg_apply(pb, w, v, y, ctx->st, &ctx->launches);
  };
  double ex = 0.0;
  CK(solve_pcg_factor(ctx->F, ctx->x, c.cg_tol, c.cg_maxit, c.solver == VMC_SOLVER_CHOLESKY_TC,
                      apply, w.r, w.z, w.p, w.q, ctx->sw, ctx->status, ctx->st, &ctx->launches,
                      iters, &ex, rel), "pcg");
  if (rel_ex) *rel_ex = ex;
  vmc_status s = check_status(ctx, "solve");
  if (s) return s;
  if (!(*rel <= c.cg_tol) || !(ex == ex))
    return fail(ctx, VMC_ERR_NUMERIC, "preconditioned CG did not reach the tolerance");
  return VMC_OK;
}

static vmc_status sample_step_set(vmc_ctx* ctx, LatticeState& L, int lattice, uint64_t* steps_out) {
  const vmc_config& c = ctx->cfg;
  SampleArgs A{};
  A.rbm = rbm_of(L);
  A.lat = lat_of(L);
  A.chains = L.chains;
  A.C = c.n_chains;
  A.L = c.sweep_len > 0 ? c.sweep_len : L.N;
  A.seed = c.seed;
  A.stream = (uint64_t)lattice;
  A.sweep0 = L.sweep;
  A.n_therm = L.thermalized ? 0 : c.therm_sweeps;
  A.n_samples = c.samples_per_chain;
  A.sweeps_per_sample = c.sweeps_per_sample;
  A.spins_out = ctx->s_spins;
  A.logpsi_out = nullptr;
  A.eloc_out = ctx->s_E;
  A.t_out = ctx->s_T;
  A.n_accept = ctx->n_accept;
  A.status = ctx->status;
  // theta of the chains' spins as one tiled product (bit-identical to the sampler's own
  // per-chain formation, which would read W once per chain).  It goes into the t buffer: a
  // chain reads its row before it writes its first record there.
  CK(theta_of(ctx, L, L.chains, c.n_chains, ctx->s_T), "theta");
  ++ctx->launches;
  A.theta_in = ctx->s_T;
  CK(launch_sample(A, ctx->st), "sample");
  ++ctx->launches;
  *steps_out = (uint64_t)(A.n_therm + A.n_samples * A.sweeps_per_sample) * (uint64_t)A.L;
  L.sweep += (uint64_t)A.n_therm + (uint64_t)A.n_samples * A.sweeps_per_sample;
  L.thermalized = true;
  return VMC_OK;
}

// One SR step; `given` (dev int8 [Ns][N]) replaces the sampling by a given sample set.
static vmc_status sr_step_impl(vmc_ctx* ctx, int lattice, double dt, vmc_sr_stats* stats,
                               const int8_t* given) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  LatticeState& L = ctx->lats[lattice];
  const vmc_config& c = ctx->cfg;
  const int64_t Ns = ctx->Ns;
  const int64_t launches0 = ctx->launches;
  CK(cudaMemsetAsync(ctx->n_accept, 0, sizeof(unsigned long long), ctx->st), "sr_step");
  CK(cudaEventRecord(ctx->ev[0], ctx->st), "sr_step");
  // 1. sample Ns configurations; E_loc and tanh(theta) fused at every record point (or take
  //    the given configurations and form both for them)
  uint64_t steps = 0;
  if (given) {
    CK(cudaMemcpyAsync(ctx->s_spins, given, (size_t)Ns * L.N, cudaMemcpyDeviceToDevice, ctx->st),
       "sr_step");
    CK(launch_theta_tanh(rbm_of(L), ctx->s_spins, Ns, ctx->s_T, ctx->st), "theta_tanh");
    CK(launch_eloc(rbm_of(L), lat_of(L), ctx->s_spins, Ns, ctx->s_E, ctx->status, ctx->st),
       "eloc");
    ctx->launches += 2;
  } else if ((s = sample_step_set(ctx, L, lattice, &steps))) {
    return s;
  }
  CK(cudaEventRecord(ctx->ev[1], ctx->st), "sr_step");
  // 2. energy statistics, <O>, F (the b- and W-block factors come from the sampler)
  CK(launch_estats(ctx->s_E, Ns, ctx->estats, ctx->status, ctx->st), "estats");
  ++ctx->launches;
  CK(cudaEventRecord(ctx->ev[2], ctx->st), "sr_step");
  int iters = 0;
  double rel = 0.0, rel_ex = NAN;
  bool converged = true;
  if (ctx->dense) {
    // 3. S (moments + centred X + Gram); with the tensor-core Gram and a mixed solver the
    //    Gram writes the solver's inputs directly
    const bool fused = c.precision == VMC_PREC_BF16SPLIT &&
                       (c.solver == VMC_SOLVER_CHOLESKY_MIXED || c.solver == VMC_SOLVER_CHOLESKY_TC);
    ctx->sw.P = L.P;
    if ((s = qfm_core(ctx, L, ctx->s_spins, ctx->s_E, Ns, c.precision, fused ? nullptr : ctx->S,
                      true, fused)))
      return s;
    CK(cudaEventRecord(ctx->ev[3], ctx->st), "sr_step");
    // 4. solve (synchronises).  The three-product BF16 split can leave S indefinite by up
    //    to the dropped lo.lo^T term; if the shifted matrix then has a non-positive pivot,
    //    S is formed again with the fourth product (PSD) and the solve repeated once.
    s = step_solve(ctx, L, fused, &iters, &rel, &rel_ex);
    if (s == VMC_ERR_NUMERIC && c.precision == VMC_PREC_BF16SPLIT) {
      if ((s = qfm_core(ctx, L, ctx->s_spins, ctx->s_E, Ns, c.precision, fused ? nullptr : ctx->S,
                        true, fused, true)))
        return s;
      ++ctx->psd_retries;
      s = step_solve(ctx, L, fused, &iters, &rel, &rel_ex);
    }
    if (s) return s;
  } else {
    // 3. <O>, F and diag(S) (S itself is never formed); on the tensor-core path <O> and F
    //    come from the same O^H u product the CG uses
    CgProblem pb{ctx->s_spins, ctx->s_T, Ns, L.N, L.M, ctx->meanO,
                 ctx->cg.Sb != nullptr && cg_tc_shape(L.N, L.M, Ns).ok, ctx->status};
    if (pb.tc) {
      CK(cg_moments_tc(pb, ctx->s_E, ctx->estats, ctx->meanO, ctx->F, ctx->cg, ctx->st,
                       &ctx->launches), "moments");
    } else {
      CK(launch_moments(ctx->s_spins, ctx->s_T, ctx->s_E, ctx->estats, Ns, L.N, L.M, ctx->partial,
                        ctx->meanO, ctx->F, ctx->st), "moments");
      ctx->launches += 2;
    }
    CK(cg_prepare(pb, ctx->cg, c.shift, c.shift_mode, ctx->st, &ctx->launches, pb.tc),
       "cg_prepare");
    cudaEventRecord(ctx->ev[6], ctx->st);
    cudaEventRecord(ctx->ev[7], ctx->st);
    CK(cudaEventRecord(ctx->ev[3], ctx->st), "sr_step");
    // 4. matrix-free CG (synchronises once per iteration)
    CK(cg_solve(pb, ctx->F, ctx->x, c.cg_tol, c.cg_maxit, ctx->cg, ctx->st, &ctx->launches, &iters,
                &rel), "cg_solve");
    if ((s = check_status(ctx, "cg"))) return s;
    if (!(rel == rel)) return fail(ctx, VMC_ERR_NUMERIC, "CG produced a non-finite residual");
    // an iterate that did not reach cg_tol is not applied (section "Diagonal shift": the
    // update is the solution of the shifted equation, not an approximation of unknown quality)
    converged = rel <= c.cg_tol;
  }
  CK(cudaEventRecord(ctx->ev[4], ctx->st), "sr_step");
  // 5. Euler update of the FP64 master parameters, refresh the FP32 copies
  if (converged) {
    CK(launch_update(L.params, ctx->x, L.P, dt, ctx->st), "update");
    L.chain_cache = false;
    ++ctx->launches;
    if ((s = refresh_fp32(ctx, L))) return s;
  }
  CK(cudaEventRecord(ctx->ev[5], ctx->st), "sr_step");
  double es[4];
  unsigned long long acc = 0;
  CK(cudaMemcpyAsync(es, ctx->estats, sizeof(es), cudaMemcpyDeviceToHost, ctx->st), "sr_step");
  CK(cudaMemcpyAsync(&acc, ctx->n_accept, sizeof(acc), cudaMemcpyDeviceToHost, ctx->st), "sr_step");
  if ((s = check_status(ctx, "sr_step"))) return s;
  if (stats) {
    stats->e_mean_re = es[0];
    stats->e_mean_im = es[1];
    stats->e_var = es[2];
    stats->e_stderr = es[3];
    stats->n_samples = Ns;
    stats->acceptance = steps ? (double)acc / ((double)steps * c.n_chains) : 0.0;
    stats->solver_iters = iters;
    stats->solver_relres = rel;
    float t[5];
    for (int k = 0; k < 5; ++k) cudaEventElapsedTime(&t[k], ctx->ev[k], ctx->ev[k + 1]);
    stats->ms_sample = t[0];
    stats->ms_grad = t[1];
    stats->ms_qfm = t[2];
    stats->ms_solve = t[3];
    stats->ms_update = t[4];
    cudaEventElapsedTime(&stats->ms_gram, ctx->ev[6], ctx->ev[7]);
    stats->launches = ctx->launches - launches0;
    stats->solver_converged = converged ? 1 : 0;
    stats->solver_relres_explicit = rel_ex == rel_ex ? rel_ex : rel;
  }
  if (!converged)
    return fail(ctx, VMC_ERR_NUMERIC, "CG did not reach cg_tol within cg_maxit iterations; "
                                      "the parameters were not updated");
  return VMC_OK;
}

vmc_status vmc_sr_step(vmc_ctx* ctx, int lattice, double dt, vmc_sr_stats* stats) {
  return sr_step_impl(ctx, lattice, dt, stats, nullptr);
}

vmc_status vmc_sr_step_on(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, double dt,
                          vmc_sr_stats* stats) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (!spins || n != ctx->Ns)
    return fail(ctx, VMC_ERR_ARG, "vmc_sr_step_on: n must equal n_chains * samples_per_chain");
  return sr_step_impl(ctx, lattice, dt, stats, spins);
}


// ---------------------------------------------------------------------------------------
// TDVP (sections "Unitary dynamics", "Regularization...", "Utilities")
// ---------------------------------------------------------------------------------------
static vmc_status tdvp_opts_ok(vmc_ctx* ctx, const vmc_tdvp_opts* o) {
  if (!o) return fail(ctx, VMC_ERR_ARG, "NULL options");
  if (!(o->eps_pinv >= 0.0) || !(o->eps_snr >= 0.0) || !(o->shift >= 0.0) ||
      (o->pinv_soft != 0 && o->pinv_soft != 1) || (o->exact != 0 && o->exact != 1) ||
      o->jacobi_max_sweeps < 0 || o->max_retries < 0 || !std::isfinite(o->gamma_re) ||
      !std::isfinite(o->gamma_im))
    return fail(ctx, VMC_ERR_ARG, "bad TDVP options");
  return VMC_OK;
}

// The regularised solve on a prepared sample set: spins sp [n][N], t = tanh theta in
// ctx->s_T, energies E, normalised weights w (null: uniform), per-sample O factor osc (may
// be null).  snr: SNR damping allowed (Monte Carlo samples), n_eff its sample count.
static vmc_status tdvp_core(vmc_ctx* ctx, LatticeState& L, const int8_t* sp, const float2* E,
                            const double* w, const float2* osc, int64_t n, bool snr,
                            const vmc_tdvp_opts& o, double2* out, bool save_S0,
                            vmc_tdvp_stats* st, const float* Od = nullptr, int64_t Pd = 0) {
  TdvpWork& tw = ctx->tw;
  const int64_t P = Od ? Pd : L.P;
  CK(tdvp_moments(sp, ctx->s_T, E, w, osc, n, L.N, L.M, tw, ctx->st, Od, Pd), "tdvp_moments");
  if (st) cudaEventRecord(ctx->ev[2], ctx->st);
  CK(tdvp_gram(sp, ctx->s_T, E, w, osc, n, L.N, L.M, tw, ctx->st, Od, Pd), "tdvp_gram");
  if (st) cudaEventRecord(ctx->ev[3], ctx->st);
  ctx->launches += 5;
  if (o.shift > 0.0) {
    CK(tdvp_shift(tw, P, o.shift, ctx->st), "tdvp_shift");
    ++ctx->launches;
  }
  if (save_S0) CK(cudaMemcpyAsync(tw.S0, tw.S, sizeof(double2) * P * P, cudaMemcpyDeviceToDevice,
                                  ctx->st), "tdvp_S0");
  if (st) cudaEventRecord(ctx->ev[4], ctx->st);
  CK(tdvp_eig(tw, P, o.jacobi_max_sweeps > 0 ? o.jacobi_max_sweeps : 40, 1e-14, ctx->st), "jacobi");
  if (st) cudaEventRecord(ctx->ev[5], ctx->st);
  const bool use_snr = o.eps_snr > 0.0 && snr;
  CK(tdvp_solve(tw, P, use_snr, o.eps_pinv, o.pinv_soft, o.eps_snr, (double)n, o.gamma_re,
                o.gamma_im, out, ctx->st), "tdvp_solve");
  ctx->launches += 4;
  if (st) {
    double es[4], ls[4], info[2];
    CK(cudaMemcpyAsync(es, tw.estats, sizeof(es), cudaMemcpyDeviceToHost, ctx->st), "tdvp");
    CK(cudaMemcpyAsync(ls, tw.lstats, sizeof(ls), cudaMemcpyDeviceToHost, ctx->st), "tdvp");
    CK(cudaMemcpyAsync(info, tw.info, sizeof(info), cudaMemcpyDeviceToHost, ctx->st), "tdvp");
    CK(cudaStreamSynchronize(ctx->st), "tdvp");
    st->e_mean_re = es[0];
    st->e_mean_im = es[1];
    st->e_var = es[2];
    st->e_stderr = es[3];
    st->lam_max = ls[0];
    st->lam_min = ls[1];
    st->kept = (int)ls[2];
    st->snr_min = ls[3];
    st->jacobi_sweeps = (int)info[0];
    st->jacobi_off = info[1];
    cudaEventElapsedTime(&st->ms_gram, ctx->ev[2], ctx->ev[3]);
    cudaEventElapsedTime(&st->ms_eig, ctx->ev[4], ctx->ev[5]);
  }
  return VMC_OK;
}

// The sample set of a right-hand side into ctx->s_spins / s_T / s_E (and Born weights in
// tw.w for exact enumeration): the caller's spins (t and E_loc formed here), all 2^N basis
// states (exact), or Ns Metropolis samples of the lattice's chains.  *w_out: normalised
// weights or null (uniform).
static vmc_status tdvp_samples(vmc_ctx* ctx, int lattice, LatticeState& L, const int8_t* spins,
                               int64_t* n, const double* w_in, bool exact, const int8_t** sp_out,
                               const double** w_out) {
  TdvpWork& tw = ctx->tw;
  const int8_t* sp = spins;
  const double* wp = nullptr;
  bool have_tE = false;
  if (sp) {
    if (w_in) {
      CK(launch_normalize_weights(w_in, *n, tw.w, ctx->status, ctx->st), "weights");
      ++ctx->launches;
      wp = tw.w;
    }
  } else if (exact) {
    if (L.N > 24 || (1ll << L.N) > ctx->Ns)
      return fail(ctx, VMC_ERR_ARG, "exact sums need 2^N <= Ns (N <= 24)");
    *n = 1ll << L.N;
    CK(launch_enum_states(ctx->s_spins, L.N, *n, ctx->st), "enum_states");
    CK(launch_logpsi(rbm_of(L), ctx->s_spins, *n, tw.lp, ctx->status, ctx->st), "logpsi");
    CK(launch_born_weights(tw.lp, *n, tw.w, ctx->status, ctx->st), "born_weights");
    ctx->launches += 3;
    wp = tw.w;
    sp = ctx->s_spins;
  } else {
    uint64_t steps = 0;
    vmc_status s = sample_step_set(ctx, L, lattice, &steps);
    if (s) return s;
    *n = ctx->Ns;
    have_tE = true;
    sp = ctx->s_spins;
  }
  if (!have_tE) {
    CK(launch_theta_tanh(rbm_of(L), sp, *n, ctx->s_T, ctx->st), "theta_tanh");
    CK(launch_eloc(rbm_of(L), lat_of(L), sp, *n, ctx->s_E, ctx->status, ctx->st), "eloc");
    ctx->launches += 2;
  }
  *sp_out = sp;
  *w_out = wp;
  return VMC_OK;
}

// thetadot of the lattice's current parameters into `out` (dev [P]) on the sample set of
// tdvp_samples.  save_S0 keeps a copy of S for the Fisher norm.
static vmc_status tdvp_eval(vmc_ctx* ctx, int lattice, LatticeState& L, const int8_t* spins,
                            int64_t n, const double* w, const vmc_tdvp_opts& o, double2* out,
                            bool save_S0, vmc_tdvp_stats* st) {
  const int8_t* sp = nullptr;
  const double* wp = nullptr;
  vmc_status s = tdvp_samples(ctx, lattice, L, spins, &n, w, o.exact != 0, &sp, &wp);
  if (s) return s;
  return tdvp_core(ctx, L, sp, ctx->s_E, wp, nullptr, n, wp == nullptr, o, out, save_S0, st);
}

vmc_status vmc_tdvp_rhs(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n,
                        const double* weights, const vmc_tdvp_opts* opts, double* thetadot,
                        vmc_tdvp_stats* stats) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if ((s = tdvp_opts_ok(ctx, opts))) return s;
  if (!ctx->cfg.tdvp) return fail(ctx, VMC_ERR_STATE, "context was created without TDVP workspaces");
  if (!thetadot) return fail(ctx, VMC_ERR_ARG, "NULL output");
  if (spins && (n < 1 || n > ctx->Ns)) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  CK(cudaEventRecord(ctx->ev[0], ctx->st), "tdvp_rhs");
  vmc_tdvp_stats local{};
  if ((s = tdvp_eval(ctx, lattice, L, spins, n, spins ? weights : nullptr, *opts,
                     reinterpret_cast<double2*>(thetadot), false, &local)))
    return s;
  CK(cudaEventRecord(ctx->ev[1], ctx->st), "tdvp_rhs");
  if ((s = check_status(ctx, "tdvp_rhs"))) return s;
  local.rhs_evals = 1;
  cudaEventElapsedTime(&local.ms, ctx->ev[0], ctx->ev[1]);
  if (stats) *stats = local;
  return VMC_OK;
}

// the lattice's parameters := y (FP64 master), FP32 copies and move tables refreshed
static vmc_status tdvp_set_params(vmc_ctx* ctx, LatticeState& L, const double2* y) {
  CK(cudaMemcpyAsync(L.params, y, sizeof(double2) * L.P, cudaMemcpyDeviceToDevice, ctx->st),
     "tdvp_params");
  L.chain_cache = false;
  return refresh_fp32(ctx, L);
}

vmc_status vmc_tdvp_step(vmc_ctx* ctx, int lattice, const vmc_tdvp_opts* opts, double* t,
                         double* tau, vmc_tdvp_stats* stats) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if ((s = tdvp_opts_ok(ctx, opts))) return s;
  if (!ctx->cfg.tdvp) return fail(ctx, VMC_ERR_STATE, "context was created without TDVP workspaces");
  if (!t || !tau || !(*tau > 0.0) || !(opts->eps_step > 0.0) || !(opts->tau_max >= 0.0))
    return fail(ctx, VMC_ERR_ARG, "bad step arguments");
  LatticeState& L = ctx->lats[lattice];
  TdvpWork& tw = ctx->tw;
  const vmc_tdvp_opts& o = *opts;
  const int64_t P = L.P;
  const double tmax = o.tau_max > 0.0 ? o.tau_max : INFINITY;
  double2 *y0 = tw.vec[0], *k1 = tw.vec[1], *k2 = tw.vec[2], *g1 = tw.vec[3], *g2 = tw.vec[4],
          *ytmp = tw.vec[5], *yfull = tw.vec[6], *yh = tw.vec[7];
  CK(cudaEventRecord(ctx->ev[0], ctx->st), "tdvp_step");
  CK(cudaMemcpyAsync(y0, L.params, sizeof(double2) * P, cudaMemcpyDeviceToDevice, ctx->st), "tdvp_step");
  vmc_tdvp_stats local{};
  if ((s = tdvp_eval(ctx, lattice, L, nullptr, 0, nullptr, o, k1, true, &local))) return s;
  int evals = 1;
  double h = std::min(*tau, tmax);
  auto eval_at = [&](const double2* y, double2* out) -> vmc_status {
    vmc_status r = tdvp_set_params(ctx, L, y);
    if (r) return r;
    ++evals;
    return tdvp_eval(ctx, lattice, L, nullptr, 0, nullptr, o, out, false, nullptr);
  };
  const int max_retries = o.max_retries > 0 ? o.max_retries : 50;
  for (int retry = 0; retry <= max_retries; ++retry) {
    // one step of size h: y_full = y0 + h/2 (k1 + f(y0 + h k1))
    CK(launch_axpy2(y0, h, k1, 0.0, nullptr, P, ytmp, ctx->st), "axpy");
    if ((s = eval_at(ytmp, k2))) return s;
    CK(launch_axpy2(y0, 0.5 * h, k1, 0.5 * h, k2, P, yfull, ctx->st), "axpy");
    // two steps of size h/2
    CK(launch_axpy2(y0, 0.5 * h, k1, 0.0, nullptr, P, ytmp, ctx->st), "axpy");
    if ((s = eval_at(ytmp, k2))) return s;
    CK(launch_axpy2(y0, 0.25 * h, k1, 0.25 * h, k2, P, yh, ctx->st), "axpy");
    if ((s = eval_at(yh, g1))) return s;
    CK(launch_axpy2(yh, 0.5 * h, g1, 0.0, nullptr, P, ytmp, ctx->st), "axpy");
    if ((s = eval_at(ytmp, g2))) return s;
    CK(launch_axpy2(yh, 0.25 * h, g1, 0.25 * h, g2, P, ytmp, ctx->st), "axpy");   // y_half
    ctx->launches += 7;
    // delta = (1/P) sqrt((y_full - y_half)^H S0 (y_full - y_half))
    int np = 0;
    CK(launch_quad_form(tw.S0, yfull, ytmp, P, tw.qpart, &np, ctx->st), "quad_form");
    ++ctx->launches;
    std::vector<double> qp(np);
    CK(cudaMemcpyAsync(qp.data(), tw.qpart, sizeof(double) * np, cudaMemcpyDeviceToHost, ctx->st),
       "quad_form");
    if ((s = check_status(ctx, "tdvp_step"))) return s;
    double q = 0.0;
    for (double v : qp) q += v;
    const double delta = std::sqrt(std::max(q, 0.0)) / (double)P;
    if (!std::isfinite(delta)) {
      tdvp_set_params(ctx, L, y0);
      return fail(ctx, VMC_ERR_NUMERIC, "TDVP step: non-finite error estimate");
    }
    double hn = delta > 0.0 ? h * std::cbrt(o.eps_step / delta) : tmax;
    if (!std::isfinite(hn)) hn = tmax;
    hn = std::min(hn, tmax);
    if (delta <= o.eps_step) {
      if ((s = tdvp_set_params(ctx, L, ytmp))) return s;
      CK(cudaEventRecord(ctx->ev[1], ctx->st), "tdvp_step");
      if ((s = check_status(ctx, "tdvp_step"))) return s;
      *t += h;
      *tau = hn;
      local.tau_used = h;
      local.tau_next = hn;
      local.delta = delta;
      local.retries = retry;
      local.rhs_evals = evals;
      cudaEventElapsedTime(&local.ms, ctx->ev[0], ctx->ev[1]);
      if (stats) *stats = local;
      return VMC_OK;
    }
    h = hn;
  }
  tdvp_set_params(ctx, L, y0);
  return fail(ctx, VMC_ERR_NUMERIC, "TDVP step: no step accepted within max_retries");
}

// ---------------------------------------------------------------------------------------
// excited states by projection (section "Finding low-energy states")
// ---------------------------------------------------------------------------------------
static vmc_status excited_ok(vmc_ctx* ctx, int lattice, int ref) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if ((s = lattice_ok(ctx, ref))) return s;
  if (ref == lattice) return fail(ctx, VMC_ERR_ARG, "the reference lattice must differ");
  if (!ctx->cfg.tdvp) return fail(ctx, VMC_ERR_STATE, "context was created without TDVP workspaces");
  const LatticeState &L = ctx->lats[lattice], &R = ctx->lats[ref];
  if (L.N != R.N || L.M != R.M) return fail(ctx, VMC_ERR_ARG, "lattices of different size");
  return VMC_OK;
}

// lambda (exp(m) mu, in tw.olap) from samples of |phi|^2
static vmc_status excited_lambda_dev(vmc_ctx* ctx, LatticeState& L, LatticeState& R, int ref,
                                     const int8_t* spins, int64_t n, bool exact) {
  TdvpWork& tw = ctx->tw;
  const int8_t* sp = spins;
  const double* w = nullptr;
  if (!sp) {
    if (exact) {
      if (L.N > 24 || (1ll << L.N) > ctx->Ns)
        return fail(ctx, VMC_ERR_ARG, "exact sums need 2^N <= Ns (N <= 24)");
      n = 1ll << L.N;
      CK(launch_enum_states(ctx->s_spins, L.N, n, ctx->st), "enum_states");
      CK(launch_logpsi(rbm_of(R), ctx->s_spins, n, tw.lp2, ctx->status, ctx->st), "logpsi");
      CK(launch_born_weights(tw.lp2, n, tw.wraw, ctx->status, ctx->st), "born_weights");
      ctx->launches += 3;
      w = tw.wraw;
    } else {
      uint64_t steps = 0;
      vmc_status s = sample_step_set(ctx, R, ref, &steps);
      if (s) return s;
      n = ctx->Ns;
    }
    sp = ctx->s_spins;
  }
  if (!w) {
    CK(launch_logpsi(rbm_of(R), sp, n, tw.lp2, ctx->status, ctx->st), "logpsi");
    ++ctx->launches;
  }
  CK(launch_logpsi(rbm_of(L), sp, n, tw.lp, ctx->status, ctx->st), "logpsi");
  CK(launch_excited_lambda(tw.lp, tw.lp2, w, n, tw.olap, ctx->status, ctx->st), "lambda");
  ctx->launches += 2;
  return VMC_OK;
}

static vmc_status excited_lambda_host(vmc_ctx* ctx, double* lam) {
  double o[3];
  CK(cudaMemcpyAsync(o, ctx->tw.olap, sizeof(o), cudaMemcpyDeviceToHost, ctx->st), "lambda");
  vmc_status s = check_status(ctx, "lambda");
  if (s) return s;
  const double e = std::exp(o[0]);
  lam[0] = e * o[1];
  lam[1] = e * o[2];
  return VMC_OK;
}

// thetadot of Psi into out, on samples of |psi|^2 (caller's, Metropolis, or all states)
static vmc_status excited_eval(vmc_ctx* ctx, int lattice, LatticeState& L, LatticeState& R,
                               const int8_t* spins, int64_t n, const vmc_tdvp_opts& o,
                               double2* out, vmc_excited_stats* st) {
  TdvpWork& tw = ctx->tw;
  const int8_t* sp = nullptr;
  const double* pw = nullptr;
  vmc_status s = tdvp_samples(ctx, lattice, L, spins, &n, nullptr, o.exact != 0, &sp, &pw);
  if (s) return s;
  CK(launch_logpsi(rbm_of(L), sp, n, tw.lp, ctx->status, ctx->st), "logpsi");
  CK(launch_logpsi(rbm_of(R), sp, n, tw.lp2, ctx->status, ctx->st), "logpsi");
  CK(launch_eloc(rbm_of(R), lat_of(L), sp, n, tw.e2, ctx->status, ctx->st), "eloc");
  CK(launch_excited_prep(tw.lp, tw.lp2, ctx->s_E, tw.e2, pw, tw.olap, n, tw.osc, tw.wraw, tw.eexc,
                         ctx->st), "excited_prep");
  CK(launch_normalize_weights(tw.wraw, n, tw.w, ctx->status, ctx->st, tw.olap + 4), "weights");
  ctx->launches += 5;
  vmc_tdvp_stats ts{};
  if ((s = tdvp_core(ctx, L, sp, tw.eexc, tw.w, tw.osc, n, false, o, out, false,
                     st ? &ts : nullptr)))
    return s;
  if (st) {
    double o6[6];
    CK(cudaMemcpyAsync(o6, tw.olap, sizeof(o6), cudaMemcpyDeviceToHost, ctx->st), "excited");
    CK(cudaStreamSynchronize(ctx->st), "excited");
    const double e = std::exp(o6[0]);
    st->lambda_re = e * o6[1];
    st->lambda_im = e * o6[2];
    st->ess = o6[5] > 0.0 ? o6[4] * o6[4] / o6[5] : 0.0;
    st->tdvp = ts;
  }
  return VMC_OK;
}

vmc_status vmc_excited_lambda(vmc_ctx* ctx, int lattice, int ref_lattice, const int8_t* spins_phi,
                              int64_t n, int exact, double* lambda_out) {
  vmc_status s = excited_ok(ctx, lattice, ref_lattice);
  if (s) return s;
  if (!lambda_out || (spins_phi && (n < 1 || n > ctx->Ns)) || (exact != 0 && exact != 1))
    return fail(ctx, VMC_ERR_ARG, "bad arguments");
  if ((s = excited_lambda_dev(ctx, ctx->lats[lattice], ctx->lats[ref_lattice], ref_lattice,
                              spins_phi, n, exact != 0)))
    return s;
  return excited_lambda_host(ctx, lambda_out);
}

vmc_status vmc_excited_rhs(vmc_ctx* ctx, int lattice, int ref_lattice, const int8_t* spins_psi,
                           int64_t n, const double* lambda, const vmc_tdvp_opts* opts,
                           double* thetadot, vmc_excited_stats* stats) {
  vmc_status s = excited_ok(ctx, lattice, ref_lattice);
  if (s) return s;
  if ((s = tdvp_opts_ok(ctx, opts))) return s;
  if (!thetadot || (spins_psi && (n < 1 || n > ctx->Ns))) return fail(ctx, VMC_ERR_ARG, "bad arguments");
  if (lambda) {
    const double o[3] = {0.0, lambda[0], lambda[1]};
    CK(cudaMemcpyAsync(ctx->tw.olap, o, sizeof(o), cudaMemcpyHostToDevice, ctx->st), "lambda");
    CK(cudaStreamSynchronize(ctx->st), "lambda");
  }
  CK(cudaEventRecord(ctx->ev[0], ctx->st), "excited_rhs");
  vmc_excited_stats local{};
  if ((s = excited_eval(ctx, lattice, ctx->lats[lattice], ctx->lats[ref_lattice], spins_psi, n,
                        *opts, reinterpret_cast<double2*>(thetadot), &local)))
    return s;
  CK(cudaEventRecord(ctx->ev[1], ctx->st), "excited_rhs");
  if ((s = check_status(ctx, "excited_rhs"))) return s;
  local.tdvp.rhs_evals = 1;
  cudaEventElapsedTime(&local.tdvp.ms, ctx->ev[0], ctx->ev[1]);
  if (stats) *stats = local;
  return VMC_OK;
}

vmc_status vmc_excited_step(vmc_ctx* ctx, int lattice, int ref_lattice, double dt,
                            const vmc_tdvp_opts* opts, vmc_excited_stats* stats) {
  vmc_status s = excited_ok(ctx, lattice, ref_lattice);
  if (s) return s;
  if ((s = tdvp_opts_ok(ctx, opts))) return s;
  if (!std::isfinite(dt)) return fail(ctx, VMC_ERR_ARG, "bad dt");
  LatticeState &L = ctx->lats[lattice], &R = ctx->lats[ref_lattice];
  TdvpWork& tw = ctx->tw;
  CK(cudaEventRecord(ctx->ev[0], ctx->st), "excited_step");
  if ((s = excited_lambda_dev(ctx, L, R, ref_lattice, nullptr, 0, opts->exact != 0))) return s;
  vmc_excited_stats local{};
  if ((s = excited_eval(ctx, lattice, L, R, nullptr, 0, *opts, tw.vec[1], &local))) return s;
  // theta <- theta + dt thetadot (thetadot = -S^+ F: the SR step of Psi)
  CK(launch_axpy2(L.params, dt, tw.vec[1], 0.0, nullptr, L.P, tw.vec[0], ctx->st), "axpy");
  if ((s = tdvp_set_params(ctx, L, tw.vec[0]))) return s;
  CK(cudaEventRecord(ctx->ev[1], ctx->st), "excited_step");
  if ((s = check_status(ctx, "excited_step"))) return s;
  local.tdvp.rhs_evals = 1;
  cudaEventElapsedTime(&local.tdvp.ms, ctx->ev[0], ctx->ev[1]);
  if (stats) *stats = local;
  return VMC_OK;
}

// ---------------------------------------------------------------------------------------
// the autoregressive network as the ansatz (section "Autoregressive neural quantum states")
// ---------------------------------------------------------------------------------------
static vmc_status ar_ok(vmc_ctx* ctx, int lattice) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (!ctx->cfg.ar_ansatz) return fail(ctx, VMC_ERR_STATE, "context was created without ar_ansatz");
  return VMC_OK;
}

static MadeDev ar_dev(vmc_ctx* ctx, LatticeState& L) {
  return made_view(L.made, L.W1t, L.W2t, L.W3t, L.N, ctx->cfg.made_hidden);
}

vmc_status vmc_ar_set_params(vmc_ctx* ctx, int lattice, const double* params_host) {
  vmc_status s = ar_ok(ctx, lattice);
  if (s) return s;
  if (!params_host) return fail(ctx, VMC_ERR_ARG, "NULL parameters");
  LatticeState& L = ctx->lats[lattice];
  CK(cudaMemcpyAsync(L.ar_params, params_host, sizeof(double) * L.ar_P, cudaMemcpyHostToDevice,
                     ctx->st), "ar_set_params");
  CK(launch_to_f32(L.ar_params, L.ar_P, L.made, ctx->st), "ar_set_params");
  CK(launch_made_transpose(ar_dev(ctx, L), ctx->st), "ar_set_params");
  ctx->launches += 2;
  CK(cudaStreamSynchronize(ctx->st), "ar_set_params");
  return VMC_OK;
}

vmc_status vmc_ar_get_params(vmc_ctx* ctx, int lattice, double* params_host) {
  vmc_status s = ar_ok(ctx, lattice);
  if (s) return s;
  if (!params_host) return fail(ctx, VMC_ERR_ARG, "NULL output");
  LatticeState& L = ctx->lats[lattice];
  CK(cudaMemcpyAsync(params_host, L.ar_params, sizeof(double) * L.ar_P, cudaMemcpyDeviceToHost,
                     ctx->st), "ar_get_params");
  CK(cudaStreamSynchronize(ctx->st), "ar_get_params");
  return VMC_OK;
}

vmc_status vmc_ar_logpsi(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* logpsi) {
  vmc_status s = ar_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && (!spins || !logpsi))) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  CK(launch_made_logq(ar_dev(ctx, L), spins, n, logpsi, ctx->st), "ar_logpsi");
  CK(launch_scale_f32(logpsi, n, 0.5f, ctx->st), "ar_logpsi");
  ctx->launches += 2;
  return check_status(ctx, "ar_logpsi");
}

vmc_status vmc_ar_sample(vmc_ctx* ctx, int lattice, int64_t n, int8_t* spins_out, float* logpsi_out) {
  vmc_status s = ar_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && !spins_out)) return fail(ctx, VMC_ERR_ARG, "bad batch");
  if (n > 0 && !logpsi_out && n > ctx->Ns) return fail(ctx, VMC_ERR_ARG, "n > Ns needs logpsi_out");
  LatticeState& L = ctx->lats[lattice];
  float* lq = logpsi_out ? logpsi_out : ctx->ar_lq;
  CK(launch_made_sample(ar_dev(ctx, L), n, ctx->cfg.seed, (uint64_t)lattice, L.made_round, spins_out,
                        lq, ctx->st), "ar_sample");
  ++L.made_round;
  if (logpsi_out) CK(launch_scale_f32(logpsi_out, n, 0.5f, ctx->st), "ar_sample");
  ctx->launches += 2;
  return check_status(ctx, "ar_sample");
}

// E_loc of a batch (n <= Ns) into E; lq receives log q of the batch
static vmc_status ar_eloc_core(vmc_ctx* ctx, LatticeState& L, const int8_t* spins, int64_t n,
                               float2* E) {
  const MadeDev D = ar_dev(ctx, L);
  const LatDev lat = lat_of(L);
  const int64_t K = L.lat.model == 0 ? L.N : L.nb;
  CK(launch_ar_connected(spins, n, lat, ctx->ar_conn, ctx->st), "ar_connected");
  CK(launch_made_logq(D, ctx->ar_conn, n * K, ctx->ar_lqc, ctx->st), "ar_logq");
  CK(launch_made_logq(D, spins, n, ctx->ar_lq, ctx->st), "ar_logq");
  CK(launch_ar_eloc(spins, ctx->ar_lq, ctx->ar_lqc, n, lat, E, ctx->status, ctx->st), "ar_eloc");
  ctx->launches += 4;
  return VMC_OK;
}

vmc_status vmc_ar_local_energy(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* eloc) {
  vmc_status s = ar_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || n > ctx->Ns || (n > 0 && (!spins || !eloc))) return fail(ctx, VMC_ERR_ARG, "bad batch");
  if (n == 0) return VMC_OK;
  if ((s = ar_eloc_core(ctx, ctx->lats[lattice], spins, n, reinterpret_cast<float2*>(eloc)))) return s;
  return check_status(ctx, "ar_local_energy");
}

// <E> into ctx->estats, per-sample backward into ctx->mw, <O> and F into ctx->meanO / ctx->F
static vmc_status ar_grad_core(vmc_ctx* ctx, LatticeState& L, const int8_t* spins, const float2* E,
                               int64_t n) {
  CK(launch_estats(E, n, ctx->estats, ctx->status, ctx->st), "estats");
  CK(launch_made_fwd_bwd(ar_dev(ctx, L), spins, n, ctx->mw, ctx->st), "ar_backward");
  CK(launch_ar_moments(spins, ctx->mw, E, ctx->estats, n, L.N, ctx->cfg.made_hidden, ctx->ar_part,
                       ctx->ar_part_cap, ctx->meanO, ctx->F, ctx->st), "ar_moments");
  ctx->launches += 4;
  return VMC_OK;
}

vmc_status vmc_ar_grad(vmc_ctx* ctx, int lattice, const int8_t* spins, const float* eloc, int64_t n,
                       float* O_out, double* meanO_out, double* F_out, double* E_stats) {
  vmc_status s = ar_ok(ctx, lattice);
  if (s) return s;
  if (n < 1 || n > ctx->Ns || !spins || !eloc) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  if ((s = ar_grad_core(ctx, L, spins, reinterpret_cast<const float2*>(eloc), n))) return s;
  if (O_out) {
    CK(launch_ar_dense_o(spins, ctx->mw, n, L.N, ctx->cfg.made_hidden, O_out, ctx->st), "ar_dense_o");
    ++ctx->launches;
  }
  // <O> and F are real: copy the real parts out
  if (meanO_out)
    CK(cudaMemcpy2DAsync(meanO_out, sizeof(double), ctx->meanO, sizeof(double2), sizeof(double),
                         L.ar_P, cudaMemcpyDeviceToDevice, ctx->st), "ar_grad");
  if (F_out)
    CK(cudaMemcpy2DAsync(F_out, sizeof(double), ctx->F, sizeof(double2), sizeof(double), L.ar_P,
                         cudaMemcpyDeviceToDevice, ctx->st), "ar_grad");
  if (E_stats) CK(cudaMemcpyAsync(E_stats, ctx->estats, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                  ctx->st), "ar_grad");
  return check_status(ctx, "ar_grad");
}

vmc_status vmc_ar_sr_step(vmc_ctx* ctx, int lattice, double dt, vmc_sr_stats* stats) {
  vmc_status s = ar_ok(ctx, lattice);
  if (s) return s;
  if (!ctx->dense) return fail(ctx, VMC_ERR_STATE, "the autoregressive SR step needs a dense solver");
  LatticeState& L = ctx->lats[lattice];
  const int64_t Ns = ctx->Ns, P = L.ar_P;
  const int64_t launches0 = ctx->launches;
  CK(cudaEventRecord(ctx->ev[0], ctx->st), "ar_sr_step");
  // 1. Ns exact draws
  CK(launch_made_sample(ar_dev(ctx, L), Ns, ctx->cfg.seed, (uint64_t)lattice, L.made_round,
                        ctx->s_spins, ctx->ar_lq, ctx->st), "ar_sample");
  ++L.made_round;
  ++ctx->launches;
  CK(cudaEventRecord(ctx->ev[1], ctx->st), "ar_sr_step");
  // 2. E_loc, <E>, per-sample O, <O>, F
  if ((s = ar_eloc_core(ctx, L, ctx->s_spins, Ns, ctx->s_E))) return s;
  if ((s = ar_grad_core(ctx, L, ctx->s_spins, ctx->s_E, Ns))) return s;
  CK(cudaEventRecord(ctx->ev[2], ctx->st), "ar_sr_step");
  // 3. S = <Obar Obar^T> (FP32 SIMT Gram of the P real rows, FP64 result)
  const int64_t rows_real = (P + 127) / 128 * 128;
  if (rows_real > ctx->rows_pad || Ns > ctx->ld) return fail(ctx, VMC_ERR_ARG, "S workspace too small");
  CK(launch_ar_build_x(ctx->s_spins, ctx->mw, ctx->meanO, Ns, L.N, ctx->cfg.made_hidden,
                       rows_real, ctx->ld, ctx->X32, ctx->st), "ar_build_x");
  cudaEventRecord(ctx->ev[6], ctx->st);
  CK(launch_gram_f32(ctx->X32, rows_real, ctx->ld, P, 1.0 / (double)Ns, ctx->S, true, ctx->gpart,
                     ctx->gpart_cap, ctx->st, true), "gram_f32");
  cudaEventRecord(ctx->ev[7], ctx->st);
  CK(launch_freeze_zero_rows(ctx->S, ctx->F, P, ctx->st), "freeze");
  ctx->launches += 3;
  CK(cudaEventRecord(ctx->ev[3], ctx->st), "ar_sr_step");
  // 4. shifted solve, 5. update
  int iters = 0;
  double rel = 0.0;
  if ((s = solve_core(ctx, P, ctx->S, ctx->F, ctx->x, &iters, &rel))) return s;
  CK(cudaEventRecord(ctx->ev[4], ctx->st), "ar_sr_step");
  CK(launch_ar_update(L.ar_params, ctx->x, P, dt, L.made, ctx->st), "ar_update");
  CK(launch_made_transpose(ar_dev(ctx, L), ctx->st), "ar_update");
  ctx->launches += 2;
  CK(cudaEventRecord(ctx->ev[5], ctx->st), "ar_sr_step");
  double es[4];
  CK(cudaMemcpyAsync(es, ctx->estats, sizeof(es), cudaMemcpyDeviceToHost, ctx->st), "ar_sr_step");
  if ((s = check_status(ctx, "ar_sr_step"))) return s;
  if (stats) {
    *stats = vmc_sr_stats{};
    stats->e_mean_re = es[0];
    stats->e_mean_im = es[1];
    stats->e_var = es[2];
    stats->e_stderr = es[3];
    stats->n_samples = Ns;
    stats->acceptance = 1.0;
    stats->solver_iters = iters;
    stats->solver_relres = rel;
    stats->solver_relres_explicit = rel;
    stats->solver_converged = 1;
    float t[5];
    for (int k = 0; k < 5; ++k) cudaEventElapsedTime(&t[k], ctx->ev[k], ctx->ev[k + 1]);
    stats->ms_sample = t[0];
    stats->ms_grad = t[1];
    stats->ms_qfm = t[2];
    stats->ms_solve = t[3];
    stats->ms_update = t[4];
    cudaEventElapsedTime(&stats->ms_gram, ctx->ev[6], ctx->ev[7]);
    stats->launches = ctx->launches - launches0;
  }
  return VMC_OK;
}

// ---------------------------------------------------------------------------------------
// the translation-symmetric CNN-ELU ansatz (section "Ground state search", Eq. gs_nqs)
// ---------------------------------------------------------------------------------------
static vmc_status cnn_ok(vmc_ctx* ctx, int lattice) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (!ctx->cfg.cnn_ansatz) return fail(ctx, VMC_ERR_STATE, "context was created without cnn_ansatz");
  return VMC_OK;
}

static CnnDev cnn_dev(const LatticeState& L) { return CnnDev{L.N, L.lat.alpha, L.cnn_W, L.cnn_b}; }

vmc_status vmc_cnn_set_params(vmc_ctx* ctx, int lattice, const double* params_host) {
  vmc_status s = cnn_ok(ctx, lattice);
  if (s) return s;
  if (!params_host) return fail(ctx, VMC_ERR_ARG, "NULL parameters");
  LatticeState& L = ctx->lats[lattice];
  CK(cudaMemcpyAsync(L.cnn_params, params_host, sizeof(double) * L.cnn_P, cudaMemcpyHostToDevice,
                     ctx->st), "cnn_set_params");
  CK(launch_cnn_prep(L.cnn_params, L.lat.alpha, L.N, L.cnn_W, L.cnn_b, ctx->st), "cnn_set_params");
  ++ctx->launches;
  CK(cudaStreamSynchronize(ctx->st), "cnn_set_params");
  return VMC_OK;
}

vmc_status vmc_cnn_get_params(vmc_ctx* ctx, int lattice, double* params_host) {
  vmc_status s = cnn_ok(ctx, lattice);
  if (s) return s;
  if (!params_host) return fail(ctx, VMC_ERR_ARG, "NULL output");
  LatticeState& L = ctx->lats[lattice];
  CK(cudaMemcpyAsync(params_host, L.cnn_params, sizeof(double) * L.cnn_P, cudaMemcpyDeviceToHost,
                     ctx->st), "cnn_get_params");
  CK(cudaStreamSynchronize(ctx->st), "cnn_get_params");
  return VMC_OK;
}

vmc_status vmc_cnn_eval(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* logpsi,
                        float* eloc) {
  vmc_status s = cnn_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && (!spins || (!logpsi && !eloc)))) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  CK(launch_cnn_eval(cnn_dev(L), lat_of(L), spins, n, logpsi, reinterpret_cast<float2*>(eloc),
                     ctx->status, ctx->st), "cnn_eval");
  ++ctx->launches;
  return check_status(ctx, "cnn_eval");
}

vmc_status vmc_cnn_grad(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* O_out) {
  vmc_status s = cnn_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && (!spins || !O_out))) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  CK(launch_cnn_ok(cnn_dev(L), spins, n, O_out, ctx->st), "cnn_grad");
  ++ctx->launches;
  return check_status(ctx, "cnn_grad");
}

static vmc_status cnn_sample_core(vmc_ctx* ctx, int lattice, LatticeState& L, int n_therm,
                                  int n_samples, int8_t* spins_out, float* logpsi_out,
                                  float2* eloc_out) {
  const vmc_config& c = ctx->cfg;
  CnnSampleArgs A{};
  A.D = cnn_dev(L);
  A.lat = lat_of(L);
  A.chains = L.chains;
  A.C = c.n_chains;
  A.L = c.sweep_len > 0 ? c.sweep_len : L.N;
  A.seed = c.seed;
  A.stream = (uint64_t)lattice;
  A.sweep0 = L.cnn_sweep;
  A.n_therm = n_therm;
  A.n_samples = n_samples;
  A.sweeps_per_sample = c.sweeps_per_sample;
  A.spins_out = spins_out;
  A.logpsi_out = logpsi_out;
  A.eloc_out = eloc_out;
  A.n_accept = ctx->n_accept;
  A.status = ctx->status;
  CK(launch_cnn_sample(A, ctx->st), "cnn_sample");
  ++ctx->launches;
  L.cnn_sweep += (uint64_t)n_therm + (uint64_t)n_samples * c.sweeps_per_sample;
  L.cnn_thermalized = true;
  return VMC_OK;
}

vmc_status vmc_cnn_sample(vmc_ctx* ctx, int lattice, int n_therm, int n_samples, int8_t* spins_out,
                          float* logpsi_out, float* eloc_out) {
  vmc_status s = cnn_ok(ctx, lattice);
  if (s) return s;
  if (n_therm < 0 || n_samples < 0) return fail(ctx, VMC_ERR_ARG, "bad counts");
  if ((s = cnn_sample_core(ctx, lattice, ctx->lats[lattice], n_therm, n_samples, spins_out,
                           logpsi_out, reinterpret_cast<float2*>(eloc_out))))
    return s;
  return check_status(ctx, "cnn_sample");
}

vmc_status vmc_cnn_sr_step(vmc_ctx* ctx, int lattice, double dt, const vmc_tdvp_opts* opts,
                           vmc_tdvp_stats* stats) {
  vmc_status s = cnn_ok(ctx, lattice);
  if (s) return s;
  if ((s = tdvp_opts_ok(ctx, opts))) return s;
  if (!std::isfinite(dt)) return fail(ctx, VMC_ERR_ARG, "bad dt");
  LatticeState& L = ctx->lats[lattice];
  const vmc_config& c = ctx->cfg;
  CK(cudaEventRecord(ctx->ev[0], ctx->st), "cnn_sr_step");
  // Ns Metropolis samples with fused E_loc, then the dense log-derivatives
  if ((s = cnn_sample_core(ctx, lattice, L, L.cnn_thermalized ? 0 : c.therm_sweeps,
                           c.samples_per_chain, ctx->s_spins, nullptr, ctx->s_E)))
    return s;
  CK(launch_cnn_ok(cnn_dev(L), ctx->s_spins, ctx->Ns, ctx->cnn_O, ctx->st), "cnn_ok");
  ++ctx->launches;
  // the regularised solve (diagonal shift and pseudo-inverse of opts), then the Euler step
  vmc_tdvp_stats local{};
  if ((s = tdvp_core(ctx, L, ctx->s_spins, ctx->s_E, nullptr, nullptr, ctx->Ns, true, *opts,
                     ctx->tw.vec[1], false, &local, ctx->cnn_O, L.cnn_P)))
    return s;
  CK(launch_cnn_update(L.cnn_params, ctx->tw.vec[1], L.cnn_P, dt, ctx->st), "cnn_update");
  CK(launch_cnn_prep(L.cnn_params, L.lat.alpha, L.N, L.cnn_W, L.cnn_b, ctx->st), "cnn_update");
  ctx->launches += 2;
  CK(cudaEventRecord(ctx->ev[1], ctx->st), "cnn_sr_step");
  if ((s = check_status(ctx, "cnn_sr_step"))) return s;
  local.rhs_evals = 1;
  cudaEventElapsedTime(&local.ms, ctx->ev[0], ctx->ev[1]);
  if (stats) *stats = local;
  return VMC_OK;
}

static vmc_status made_ok(vmc_ctx* ctx, int lattice) {
  vmc_status s = lattice_ok(ctx, lattice);
  if (s) return s;
  if (ctx->cfg.made_hidden <= 0) return fail(ctx, VMC_ERR_STATE, "context has no learned proposal (made_hidden = 0)");
  return VMC_OK;
}

vmc_status vmc_made_set_params(vmc_ctx* ctx, int lattice, const float* params_host) {
  vmc_status s = made_ok(ctx, lattice);
  if (s) return s;
  if (!params_host) return fail(ctx, VMC_ERR_ARG, "params_host is NULL");
  LatticeState& L = ctx->lats[lattice];
  const int64_t np = made_nparams(L.N, ctx->cfg.made_hidden);
  CK(cudaMemcpyAsync(L.made, params_host, np * sizeof(float), cudaMemcpyHostToDevice, ctx->st), "made_set_params");
  CK(cudaMemsetAsync(L.made_m, 0, np * sizeof(float), ctx->st), "made_set_params");
  CK(cudaMemsetAsync(L.made_v, 0, np * sizeof(float), ctx->st), "made_set_params");
  CK(launch_made_transpose(made_of(ctx, L), ctx->st), "made_transpose");
  ++ctx->launches;
  L.made_t = 0;
  L.chain_cache = false;
  CK(cudaStreamSynchronize(ctx->st), "made_set_params");
  return VMC_OK;
}

vmc_status vmc_made_get_params(vmc_ctx* ctx, int lattice, float* params_host) {
  vmc_status s = made_ok(ctx, lattice);
  if (s) return s;
  if (!params_host) return fail(ctx, VMC_ERR_ARG, "params_host is NULL");
  LatticeState& L = ctx->lats[lattice];
  const int64_t np = made_nparams(L.N, ctx->cfg.made_hidden);
  CK(cudaMemcpyAsync(params_host, L.made, np * sizeof(float), cudaMemcpyDeviceToHost, ctx->st), "made_get_params");
  CK(cudaStreamSynchronize(ctx->st), "made_get_params");
  return VMC_OK;
}

vmc_status vmc_made_logq(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* logq) {
  vmc_status s = made_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && (!spins || !logq))) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  CK(launch_made_logq(made_of(ctx, L), spins, n, logq, ctx->st), "made_logq");
  ++ctx->launches;
  return VMC_OK;
}

static double mean_neg(const float* d_logq, int64_t n, vmc_ctx* ctx) {
  std::vector<float> h((size_t)n);
  cudaMemcpyAsync(h.data(), d_logq, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->st);
  cudaStreamSynchronize(ctx->st);
  double acc = 0.0;
  for (float v : h) acc -= (double)v;
  return acc / (double)n;
}

vmc_status vmc_made_grad(vmc_ctx* ctx, int lattice, const int8_t* spins, int64_t n, float* grad,
                         double* loss) {
  vmc_status s = made_ok(ctx, lattice);
  if (s) return s;
  if (n < 1 || n > ctx->made_cap || !spins || !grad) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  CK(launch_made_grad(made_of(ctx, L), spins, n, ctx->mw, grad, ctx->st), "made_grad");
  ctx->launches += 7;
  const double l = mean_neg(ctx->mw.logq, n, ctx);
  if (loss) *loss = l;
  return check_status(ctx, "made_grad");
}

vmc_status vmc_proposal_train(vmc_ctx* ctx, int lattice, const int8_t* samples, int64_t n,
                              int epochs, double lr, double* loss) {
  vmc_status s = made_ok(ctx, lattice);
  if (s) return s;
  if (n < 1 || epochs < 0 || !samples || !(lr > 0.0)) return fail(ctx, VMC_ERR_ARG, "bad training arguments");
  LatticeState& L = ctx->lats[lattice];
  const int64_t B = std::min<int64_t>(ctx->cfg.made_batch > 0 ? ctx->cfg.made_batch : 4096, ctx->made_cap);
  const int64_t np = made_nparams(L.N, ctx->cfg.made_hidden);
  MadeDev D = made_of(ctx, L);
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t b0 = 0; b0 < n; b0 += B) {
      const int64_t nb = std::min<int64_t>(B, n - b0);
      CK(launch_made_grad(D, samples + b0 * L.N, nb, ctx->mw, L.made_g, ctx->st), "made_grad");
      CK(launch_adam(L.made, L.made_m, L.made_v, L.made_g, np, ++L.made_t, (float)lr, ctx->st), "adam");
      CK(launch_made_transpose(D, ctx->st), "made_transpose");
      ctx->launches += 9;
    }
  }
  L.chain_cache = false;
  if (loss) {
    double acc = 0.0;
    for (int64_t b0 = 0; b0 < n; b0 += B) {
      const int64_t nb = std::min<int64_t>(B, n - b0);
      CK(launch_made_logq(D, samples + b0 * L.N, nb, ctx->mw.logq, ctx->st), "made_logq");
      ++ctx->launches;
      acc += mean_neg(ctx->mw.logq, nb, ctx) * (double)nb;
    }
    *loss = acc / (double)n;
  }
  return check_status(ctx, "proposal_train");
}

vmc_status vmc_made_sample(vmc_ctx* ctx, int lattice, int64_t n, uint64_t round, int8_t* spins,
                           float* logq) {
  vmc_status s = made_ok(ctx, lattice);
  if (s) return s;
  if (n < 0 || (n > 0 && !spins)) return fail(ctx, VMC_ERR_ARG, "bad batch");
  LatticeState& L = ctx->lats[lattice];
  CK(launch_made_sample(made_of(ctx, L), n, ctx->cfg.seed, (uint64_t)lattice, round, spins, logq,
                        ctx->st), "made_sample");
  ++ctx->launches;
  return VMC_OK;
}

vmc_status vmc_sample_learned(vmc_ctx* ctx, int lattice, int n_rounds, int8_t* spins_out,
                              float* eloc_out, double* acceptance) {
  vmc_status s = made_ok(ctx, lattice);
  if (s) return s;
  if (n_rounds < 0) return fail(ctx, VMC_ERR_ARG, "negative round count");
  LatticeState& L = ctx->lats[lattice];
  const int64_t C = ctx->cfg.n_chains;
  MadeDev D = made_of(ctx, L);
  if (!L.chain_cache) {
    CK(launch_logpsi(rbm_of(L), L.chains, C, L.chain_lp, ctx->status, ctx->st), "logpsi");
    CK(launch_made_logq(D, L.chains, C, L.chain_lq, ctx->st), "made_logq");
    ctx->launches += 2;
    L.chain_cache = true;
  }
  CK(cudaMemsetAsync(ctx->n_accept, 0, sizeof(unsigned long long), ctx->st), "sample_learned");
  for (int r = 0; r < n_rounds; ++r) {
    const uint64_t round = L.made_round++;
    CK(launch_made_sample(D, C, ctx->cfg.seed, (uint64_t)lattice, round, L.prop, L.prop_lq, ctx->st),
       "made_sample");
    CK(launch_logpsi(rbm_of(L), L.prop, C, L.prop_lp, ctx->status, ctx->st), "logpsi");
    CK(launch_made_mh(C, L.N, L.prop, L.prop_lp, L.prop_lq, L.chains, L.chain_lp, L.chain_lq,
                      ctx->cfg.seed, (uint64_t)lattice, round, ctx->n_accept, ctx->st), "made_mh");
    ctx->launches += 3;
    if (spins_out)
      CK(cudaMemcpyAsync(spins_out + (int64_t)r * C * L.N, L.chains, (size_t)C * L.N,
                         cudaMemcpyDeviceToDevice, ctx->st), "sample_learned");
    if (eloc_out) {
      CK(launch_eloc(rbm_of(L), lat_of(L), L.chains, C,
                     reinterpret_cast<float2*>(eloc_out) + (int64_t)r * C, ctx->status, ctx->st), "eloc");
      ++ctx->launches;
    }
  }
  unsigned long long acc = 0;
  CK(cudaMemcpyAsync(&acc, ctx->n_accept, sizeof(acc), cudaMemcpyDeviceToHost, ctx->st), "sample_learned");
  if ((s = check_status(ctx, "sample_learned"))) return s;
  if (acceptance) *acceptance = (n_rounds > 0) ? (double)acc / ((double)C * n_rounds) : 0.0;
  return VMC_OK;
}


static vmc_status batched_upload(vmc_ctx* ctx, int n_therm, int n_samples, int8_t* spins_out,
                                 float* eloc_out, int mpl) {
  const int nl = (int)ctx->lats.size();
  const int C = ctx->cfg.n_chains;
  std::vector<SampleArgs> args((size_t)nl);
  int64_t off = 0;
  for (int l = 0; l < nl; ++l) {
    LatticeState& L = ctx->lats[l];
    SampleArgs& A = args[(size_t)l];
    A = SampleArgs{};
    A.rbm = rbm_of(L);
    A.lat = lat_of(L);
    A.chains = L.chains;
    A.C = C;
    A.L = ctx->cfg.sweep_len > 0 ? ctx->cfg.sweep_len : L.N;
    A.seed = ctx->cfg.seed;
    A.stream = (uint64_t)l;
    A.sweep0 = L.sweep;
    A.n_therm = n_therm;
    A.n_samples = n_samples;
    A.sweeps_per_sample = ctx->cfg.sweeps_per_sample;
    A.spins_out = spins_out ? spins_out + off : nullptr;
    A.eloc_out = eloc_out ? reinterpret_cast<float2*>(eloc_out) + (int64_t)l * n_samples * C : nullptr;
    A.n_accept = ctx->n_accept;
    A.status = ctx->status;
    off += (int64_t)n_samples * C * L.N;
  }
  // heavy lattices first (work per chain ~ N * M)
  std::vector<int> order((size_t)nl);
  for (int l = 0; l < nl; ++l) order[(size_t)l] = l;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (int64_t)ctx->lats[x].N * ctx->lats[x].M > (int64_t)ctx->lats[y].N * ctx->lats[y].M;
  });
  CK(cudaMemcpyAsync(ctx->d_bargs, args.data(), sizeof(SampleArgs) * nl, cudaMemcpyHostToDevice, ctx->st), "sample_all");
  // work units: one warp's chains of one lattice (several chains per warp for small M)
  std::vector<int> ustart((size_t)nl + 1, 0);
  for (int o = 0; o < nl; ++o) {
    const int cpw = batched_chains_per_warp(ctx->lats[(size_t)order[(size_t)o]].M, mpl);
    ustart[(size_t)o + 1] = ustart[(size_t)o] + (C + cpw - 1) / cpw;
  }
  CK(cudaMemcpyAsync(ctx->d_order, order.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, ctx->st), "sample_all");
  CK(cudaMemcpyAsync(ctx->d_ustart, ustart.data(), sizeof(int) * (nl + 1), cudaMemcpyHostToDevice, ctx->st),
     "sample_all");
  CK(cudaStreamSynchronize(ctx->st), "sample_all");
  return VMC_OK;
}

// Autotuner: hidden slots per lane (the per-chain width, or a wider one up to twice it and at
// most 8, which puts several chains of the smaller lattices in one warp) and warps per block
// of the persistent launch, timed on one sweep of every chain, the faster of two launches
// per configuration (chains saved before and restored after each; sweep counters untouched).
static vmc_status batched_tune(vmc_ctx* ctx) {
  ctx->g_therm = -1;
  const int nl = (int)ctx->lats.size();
  const int C = ctx->cfg.n_chains;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev), "tune");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "tune");
  vmc_status s;
  size_t off = 0;
  for (auto& L : ctx->lats) {
    CK(cudaMemcpyAsync(ctx->chain_backup + off, L.chains, (size_t)C * L.N, cudaMemcpyDeviceToDevice, ctx->st), "tune");
    off += (size_t)C * L.N;
  }
  float best = 1e30f;
  // slots per lane: the per-chain width for the largest M and every instantiated width up to
  // twice it (at most 8), each putting the chains of more of the lattices several to a warp
  const int base = sample_slots_per_lane(ctx->Mmax);
  int mpls[4] = {base, 0, 0, 0}, nm = 1;
  for (int m = base + 1; m <= std::min(2 * base, 8) && nm < 4; ++m)
    if (sample_slots_per_lane(32 * m) == m) mpls[nm++] = m;
  const int cand[3] = {2, 4, 8};
  for (int im = 0; im < nm; ++im) {
   const int mpl = mpls[im];
   if ((s = batched_upload(ctx, 1, 0, nullptr, nullptr, mpl))) return s;
   for (int wpb : cand) {
    const int per_sm = batched_blocks_per_sm(mpl, wpb, ctx->Nmax);
    if (per_sm < 1) continue;
    const int grid = sms * per_sm;
    // the faster of two timed launches (the first also pays for the first use of the code)
    for (int rep = 0; rep < 2; ++rep) {
      CK(cudaEventRecord(ctx->ev[0], ctx->st), "tune");
      CK(launch_sample_batched(ctx->d_bargs, ctx->d_order, ctx->d_ustart, nl, ctx->Nmax, mpl,
                               ctx->d_counter, wpb, grid, 0, ctx->d_bargs, ctx->st), "tune");
      CK(cudaEventRecord(ctx->ev[1], ctx->st), "tune");
      CK(cudaEventSynchronize(ctx->ev[1]), "tune");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
      ctx->launches += 2;
      if (ms < best) { best = ms; ctx->tuned_wpb = wpb; ctx->tuned_grid = grid; ctx->tuned_mpl = mpl; }
      off = 0;
      for (auto& L : ctx->lats) {
        CK(cudaMemcpyAsync(L.chains, ctx->chain_backup + off, (size_t)C * L.N, cudaMemcpyDeviceToDevice, ctx->st), "tune");
        off += (size_t)C * L.N;
      }
    }
   }
  }
  CK(cudaStreamSynchronize(ctx->st), "tune");
  if (ctx->tuned_wpb == 0) return fail(ctx, VMC_ERR_CUDA, "no launch configuration fits");
  return check_status(ctx, "tune");
}

vmc_status vmc_sample_all(vmc_ctx* ctx, int n_therm, int n_samples, int8_t* spins_out,
                          float* eloc_out, int use_graph, double* ms) {
  if (!ctx) return VMC_ERR_ARG;
  if (n_therm < 0 || n_samples < 0) return fail(ctx, VMC_ERR_ARG, "negative sweep count");
  vmc_status s;
  if (ctx->tuned_wpb == 0 && (s = batched_tune(ctx))) return s;
  const int nl = (int)ctx->lats.size();
  const uint64_t adv = (uint64_t)n_therm + (uint64_t)n_samples * ctx->cfg.sweeps_per_sample;
  // a replay is valid only while the device descriptors still describe this call: same
  // arguments, and no per-lattice sampling or chain reset moved a sweep counter since
  bool same = ctx->graph_exec && ctx->g_therm == n_therm && ctx->g_samples == n_samples &&
              ctx->g_spins == spins_out && ctx->g_eloc == eloc_out && ctx->g_sweep.size() == ctx->lats.size();
  for (size_t l = 0; same && l < ctx->lats.size(); ++l) same = ctx->g_sweep[l] == ctx->lats[l].sweep;
  CK(cudaEventRecord(ctx->ev[0], ctx->st), "sample_all");
  if (use_graph && same) {
    CK(cudaGraphLaunch(ctx->graph_exec, ctx->st), "sample_all");
    ctx->launches += 2;
  } else {
    if ((s = batched_upload(ctx, n_therm, n_samples, spins_out, eloc_out, ctx->tuned_mpl))) return s;
    if (use_graph) {
      if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
      if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
      if (!ctx->cap_st) CK(cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking), "capture");
      CK(cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeThreadLocal), "capture");
      cudaError_t e = launch_sample_batched(ctx->d_bargs, ctx->d_order, ctx->d_ustart, nl, ctx->Nmax,
                                            ctx->tuned_mpl, ctx->d_counter, ctx->tuned_wpb,
                                            ctx->tuned_grid, adv, ctx->d_bargs, ctx->cap_st);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(ctx->cap_st, &g);
      if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(ctx, e, "capture"); }
      CK(e2, "capture");
      ctx->graph = g;
      CK(cudaGraphInstantiate(&ctx->graph_exec, g, 0), "instantiate");
      ctx->g_therm = n_therm;
      ctx->g_samples = n_samples;
      ctx->g_spins = spins_out;
      ctx->g_eloc = eloc_out;
      CK(cudaGraphLaunch(ctx->graph_exec, ctx->st), "sample_all");
    } else {
      ctx->g_therm = -1;  // the descriptors no longer match the captured graph
      CK(launch_sample_batched(ctx->d_bargs, ctx->d_order, ctx->d_ustart, nl, ctx->Nmax, ctx->tuned_mpl,
                               ctx->d_counter, ctx->tuned_wpb, ctx->tuned_grid, adv, ctx->d_bargs,
                               ctx->st), "sample_all");
    }
    ctx->launches += 2;
  }
  CK(cudaEventRecord(ctx->ev[1], ctx->st), "sample_all");
  ctx->g_sweep.resize(ctx->lats.size());
  for (size_t l = 0; l < ctx->lats.size(); ++l) {
    LatticeState& L = ctx->lats[l];
    L.sweep += adv;
    ctx->g_sweep[l] = L.sweep;
    if (n_therm > 0) L.thermalized = true;
    L.chain_cache = false;
  }
  if ((s = check_status(ctx, "sample_all"))) return s;
  if (ms) {
    float t = 0.f;
    cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]);
    *ms = t;
  }
  return VMC_OK;
}

int vmc_autotuned_warps_per_block(const vmc_ctx* ctx) { return ctx ? ctx->tuned_wpb : 0; }
int vmc_autotuned_slots_per_lane(const vmc_ctx* ctx) { return ctx ? ctx->tuned_mpl : 0; }


// ---- checkpoint / resume ------------------------------------------------------------------
namespace {
constexpr uint64_t kStateMagic = 0x3130315354434d56ull;   // "VMCSTO01" (little endian)

struct StateHeader {
  uint64_t magic;
  uint64_t bytes;                 // whole buffer
  int32_t n_lattices, n_chains, made_hidden, reserved;
};

struct LatticeRecord {
  int32_t N, M, model, thermalized;
  int64_t P;
  uint64_t sweep, made_round;
  int32_t made_t, reserved;
};

size_t state_bytes(const vmc_ctx* ctx) {
  size_t b = sizeof(StateHeader);
  for (const auto& L : ctx->lats) {
    b += sizeof(LatticeRecord) + (size_t)L.P * sizeof(double2) + (size_t)ctx->cfg.n_chains * L.N;
    if (ctx->cfg.made_hidden > 0) b += 3 * (size_t)made_nparams(L.N, ctx->cfg.made_hidden) * sizeof(float);
  }
  return b;
}
}  // namespace

vmc_status vmc_get_state(vmc_ctx* ctx, void* buf, size_t* len) {
  if (!ctx || !len) return VMC_ERR_ARG;
  const size_t need = state_bytes(ctx);
  if (!buf) {
    *len = need;
    return VMC_OK;
  }
  if (*len < need) return fail(ctx, VMC_ERR_ARG, "state buffer too small");
  uint8_t* p = static_cast<uint8_t*>(buf);
  StateHeader h{kStateMagic, need, (int32_t)ctx->lats.size(), ctx->cfg.n_chains,
                ctx->cfg.made_hidden, 0};
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  for (auto& L : ctx->lats) {
    LatticeRecord r{L.N, L.M, L.lat.model, L.thermalized ? 1 : 0, L.P, L.sweep, L.made_round,
                    L.made_t, 0};
    memcpy(p, &r, sizeof(r));
    p += sizeof(r);
    CK(cudaMemcpyAsync(p, L.params, (size_t)L.P * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st), "get_state");
    p += (size_t)L.P * sizeof(double2);
    CK(cudaMemcpyAsync(p, L.chains, (size_t)ctx->cfg.n_chains * L.N, cudaMemcpyDeviceToHost, ctx->st), "get_state");
    p += (size_t)ctx->cfg.n_chains * L.N;
    if (ctx->cfg.made_hidden > 0) {
      const size_t nb = (size_t)made_nparams(L.N, ctx->cfg.made_hidden) * sizeof(float);
      const float* src[3] = {L.made, L.made_m, L.made_v};
      for (const float* q : src) {
        CK(cudaMemcpyAsync(p, q, nb, cudaMemcpyDeviceToHost, ctx->st), "get_state");
        p += nb;
      }
    }
  }
  CK(cudaStreamSynchronize(ctx->st), "get_state");
  *len = need;
  return VMC_OK;
}

vmc_status vmc_set_state(vmc_ctx* ctx, const void* buf, size_t len) {
  if (!ctx || !buf) return VMC_ERR_ARG;
  if (len < sizeof(StateHeader)) return fail(ctx, VMC_ERR_ARG, "state buffer too small");
  const uint8_t* p = static_cast<const uint8_t*>(buf);
  StateHeader h;
  memcpy(&h, p, sizeof(h));
  p += sizeof(h);
  if (h.magic != kStateMagic) return fail(ctx, VMC_ERR_ARG, "not a vmc state");
  if (h.bytes != state_bytes(ctx) || len < h.bytes || h.n_lattices != (int32_t)ctx->lats.size() ||
      h.n_chains != ctx->cfg.n_chains || h.made_hidden != ctx->cfg.made_hidden)
    return fail(ctx, VMC_ERR_ARG, "state does not match this context's configuration");
  // validate every record before touching the context
  {
    const uint8_t* q = p;
    for (auto& L : ctx->lats) {
      LatticeRecord r;
      memcpy(&r, q, sizeof(r));
      if (r.N != L.N || r.M != L.M || r.model != L.lat.model || r.P != L.P)
        return fail(ctx, VMC_ERR_ARG, "state does not match this context's lattices");
      q += sizeof(r) + (size_t)L.P * sizeof(double2) + (size_t)ctx->cfg.n_chains * L.N;
      if (ctx->cfg.made_hidden > 0) q += 3 * (size_t)made_nparams(L.N, ctx->cfg.made_hidden) * sizeof(float);
    }
  }
  for (auto& L : ctx->lats) {
    LatticeRecord r;
    memcpy(&r, p, sizeof(r));
    p += sizeof(r);
    CK(cudaMemcpyAsync(L.params, p, (size_t)L.P * sizeof(double2), cudaMemcpyHostToDevice, ctx->st), "set_state");
    p += (size_t)L.P * sizeof(double2);
    CK(cudaMemcpyAsync(L.chains, p, (size_t)ctx->cfg.n_chains * L.N, cudaMemcpyHostToDevice, ctx->st), "set_state");
    p += (size_t)ctx->cfg.n_chains * L.N;
    L.sweep = r.sweep;
    L.thermalized = r.thermalized != 0;
    L.chain_cache = false;
    vmc_status s;
    if ((s = refresh_fp32(ctx, L))) return s;
    if (ctx->cfg.made_hidden > 0) {
      const size_t nb = (size_t)made_nparams(L.N, ctx->cfg.made_hidden) * sizeof(float);
      float* dst[3] = {L.made, L.made_m, L.made_v};
      for (float* q : dst) {
        CK(cudaMemcpyAsync(q, p, nb, cudaMemcpyHostToDevice, ctx->st), "set_state");
        p += nb;
      }
      CK(launch_made_transpose(made_of(ctx, L), ctx->st), "made_transpose");
      ++ctx->launches;
      L.made_t = r.made_t;
      L.made_round = r.made_round;
    }
  }
  ctx->g_therm = -1;                                  // batched descriptors are stale
  CK(cudaStreamSynchronize(ctx->st), "set_state");
  return VMC_OK;
}

vmc_status vmc_selftest_wait_timeout(vmc_ctx* ctx, int which) {
  if (!ctx || which < 0 || which > 2) return VMC_ERR_ARG;
  unsigned* word = nullptr;
  CK(cudaMalloc(&word, 4 * sizeof(unsigned)), "selftest");
  cudaError_t e = which == 0   ? launch_selftest_flag_wait(word, ctx->status, ctx->st)
                  : which == 1 ? launch_selftest_mbar_wait(ctx->status, ctx->st)
                               : launch_selftest_poll_wait(word, ctx->status, ctx->st);
  ++ctx->launches;
  vmc_status s = (e == cudaSuccess) ? check_status(ctx, "selftest") : cuda_fail(ctx, e, "selftest");
  cudaFree(word);
  return s;
}

}  // extern "C"
