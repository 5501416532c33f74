"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Sizes span several tiles and a ragged tail (M = 10, 72, 128, 512 hidden units against
32-wide warps; 2P not a multiple of the 128-row Gram tile) and include the 8x8
Heisenberg workload's shapes.
"""
import numpy as np
import pytest

import oracle
from paper_2108_03409_b300 import inputs
from paper_2108_03409_b300 import vmc

from gpu_helpers import (ELOC_PER_SITE_ABS, F_REL, INIT_SCALE_SIGMA, LOGPSI_ABS, OK_ABS, OK_REL,
                         assert_logpsi_close, context, cplx, eloc_tolerance, lattice, phase_diff,
                         s_tol_bf16, s_tol_fp32, to_dev_spins, well_conditioned)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T, H = inputs.MODEL_TFIM, inputs.MODEL_HEIS

# (model, Lx, Ly, J, h, alpha, sigma, n_samples)
CASES = [
    (T, 10, 1, 1.0, 1.0, 1, 0.01, 1024),      # 1D TFIM N=10 (all states)
    (T, 6, 6, 1.0, 3.1, 2, 0.05, 1500),       # M = 72: ragged against 32 lanes
    (H, 8, 8, 1.0, 0.0, 2, 0.01, 1200),       # 8x8 Heisenberg, Marshall phase
    (H, 4, 4, 1.0, 0.0, 2, 0.2, 2000),        # larger weights
    (H, 16, 16, 1.0, 0.0, 2, 0.01, 48),       # M = 512
]
IDS = ["tfim10", "tfim6x6", "heis8x8", "heis4x4_s0.2", "heis16x16"]


def _setup(case, seed=0):
    model, Lx, Ly, J, h, alpha, sigma, n = case
    N, M = Lx * Ly, alpha * Lx * Ly
    p = inputs.rbm_params(N, M, sigma, seed=31 + seed, marshall=(Lx, Ly) if model == H else None)
    if model == T and N == 10:
        s = oracle.all_states(N)
    else:
        s = inputs.initial_spins(model, n, N, seed=7 + seed)
    return model, Lx, Ly, J, h, alpha, N, M, p, s


@pytest.mark.parametrize("precision", [vmc.PREC_FP32, vmc.PREC_BF16SPLIT], ids=["simt", "tc"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_theta_matches_oracle(case, precision):
    """theta = b + W s (Eq. rbm_ex) against the oracle.  FP32 SIMT: the FMA chain's rounding,
    2 (N + 1) 2^-24 (|b_j| + sum_i |W_ji|).  Tensor cores: the spins are exact in BF16, each
    component of W is a BF16 hi + lo pair within 2^-18 of it, and the FP32 accumulation adds
    the same chain bound: (2^-17 + 2 (N + 2) 2^-24) (|b_j| + sum_i |W_ji|).  The batches span
    several 128-configuration tiles with a ragged tail (and M against the 64-unit tiles)."""
    model, Lx, Ly, J, h, alpha, N, M, p, s = _setup(case)
    if N == 256:
        s = inputs.initial_spins(model, 300, N, seed=11)
    n = len(s)
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=1, precision=precision,
                 solver=vmc.SOLVER_CG) as ctx:           # (no dense S at 16x16)
        vmc.vmc_set_params(ctx, 0, p)
        th = torch.zeros((n, M, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_theta(ctx, 0, to_dev_spins(s), th)
        got = cplx(th).reshape(n, M)
    ref = oracle.theta(N, M, p, s)
    mag = np.abs(p[N:N + M]) + np.abs(p[N + M:].reshape(M, N)).sum(axis=1)
    if precision == vmc.PREC_FP32:
        bound = 2 * (N + 1) * 2.0 ** -24 * mag
    else:
        bound = (2.0 ** -17 + 2 * (N + 2) * 2.0 ** -24) * mag
    err = np.abs(got - ref)
    assert np.all(err <= bound[None, :]), (err / bound[None, :]).max()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_logpsi_matches_oracle(case):
    model, Lx, Ly, J, h, alpha, N, M, p, s = _setup(case)
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=max(1, s.shape[0]),
                 solver=vmc.SOLVER_CG) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        out = torch.zeros((s.shape[0], 2), dtype=torch.float32, device="cuda")
        vmc.vmc_logpsi(ctx, 0, to_dev_spins(s), out)
        got = cplx(out)
    ref = oracle.logpsi(N, M, p, s)
    ok = well_conditioned(p, s, N, M)
    assert ok.mean() >= 0.98 and np.all(np.isfinite(got))
    assert np.all(np.abs(got.imag) <= np.pi * (1 + 1e-6))      # the phase comes reduced
    assert_logpsi_close(got[ok], ref[ok], case[6])


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_logpsi_ratios_of_connected_configurations(case):
    """Delta log psi = log psi(s') - log psi(s) between each sample and every configuration
    H connects it to (the quantity E_loc and the acceptance test are built from), at the
    absolute 1e-5 bound (real part and phase mod 2 pi), computed from two vmc_logpsi
    calls.  Samples near a node of psi (for s or any s') are excluded as above."""
    model, Lx, Ly, J, h, alpha, N, M, p, s = _setup(case)
    s = s[:min(len(s), 96)]
    sp_all, owner = [], []
    for q, c in enumerate(s):
        sp, _ = oracle.connected(model, Lx, Ly, J, h, c)
        sp_all.append(sp)
        owner.append(np.full(len(sp), q))
    sp_all = np.concatenate(sp_all)
    owner = np.concatenate(owner)
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=max(len(sp_all), len(s)),
                 solver=vmc.SOLVER_CG) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        out = torch.zeros((len(sp_all), 2), dtype=torch.float32, device="cuda")
        vmc.vmc_logpsi(ctx, 0, to_dev_spins(sp_all), out)
        got = cplx(out)
    ref = oracle.logpsi(N, M, p, sp_all)
    ok = well_conditioned(p, sp_all, N, M)
    ok_owner = np.ones(len(s), bool)
    np.logical_and.at(ok_owner, owner, ok)
    keep = ok_owner[owner]
    assert keep.mean() >= 0.9
    # entry 0 of each block is s itself (oracle.connected lists the diagonal first)
    first = np.searchsorted(owner, np.arange(len(s)))
    dgot = got - got[first][owner]
    dref = ref - ref[first][owner]
    # absolute at init-scale weights; relative to |log psi(s)| for larger ones (c13 reading)
    bound = LOGPSI_ABS * (1.0 if case[6] <= INIT_SCALE_SIGMA
                          else np.maximum(1.0, np.abs(ref[first][owner])))
    assert np.all((np.abs(dgot.real - dref.real) <= bound)[keep])
    assert np.all((phase_diff(dgot.imag, dref.imag) <= bound)[keep])


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_local_energy_matches_oracle(case):
    model, Lx, Ly, J, h, alpha, N, M, p, s = _setup(case)
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=max(1, s.shape[0]),
                 solver=vmc.SOLVER_CG) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        out = torch.zeros((s.shape[0], 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, to_dev_spins(s), out)
        got = cplx(out)
    ref = oracle.eloc(model, Lx, Ly, J, h, M, p, s)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= eloc_tolerance(model, Lx, Ly, J, h, M, p, s))
    if case[6] <= 0.05:                               # init-scale weights: the plain bound
        assert np.max(np.abs(got - ref)) / N <= ELOC_PER_SITE_ABS


@pytest.mark.parametrize("model", [T, H], ids=["tfim4x4", "heis4x4"])
def test_local_energy_log_sum_fallback_matches_oracle(model):
    """A move's factor product 1 - s t tanh D over the hidden units is the E_loc ratio's
    fast path while it stays in [1e-15, 1e15]; otherwise the kernel forms the ratio from
    the log-sum of the factors.  Real parameters (no nodes of cosh theta) with one column
    of large weights (|W_j,i0| = 0.9, b_j = 0.6, M = 64) send every move touching site i0
    through the log-sum path while the ratio itself stays moderate (|log| <= 3); both
    paths' local energies against the oracle at the FP32 bound."""
    Lx = Ly = 4
    N, M, alpha, i0 = 16, 64, 4, 5
    h = 2.0 if model == T else 0.0
    rng = np.random.default_rng(71)
    a = rng.normal(0, 0.05, N)
    b = 0.6 + rng.normal(0, 0.05, M)
    W = rng.normal(0, 0.02, (M, N))
    W[:, i0] = np.where(np.arange(M) % 2 == 0, 0.9, -0.9)
    p = np.concatenate([a, b, W.reshape(-1)]).astype(np.complex128)
    s = inputs.initial_spins(model, 400, N, seed=72)
    # host check that the log-sum path is exercised: moves whose product leaves the range
    t = np.tanh(b[None, :] + s.astype(np.float64) @ W.T)
    n_log_sum = 0
    for q in range(len(s)):
        sp, _ = oracle.connected(model, Lx, Ly, 1.0, h, s[q])
        for c in sp[1:]:
            flip = np.nonzero(c != s[q])[0]
            D = 2 * W[:, flip[0]] - (2 * W[:, flip[1]] if len(flip) == 2 else 0)
            lp = np.sum(np.log(np.abs(1 - s[q, flip[0]] * t[q] * np.tanh(D))))
            n_log_sum += abs(lp) > 15 * np.log(10)
    assert n_log_sum >= len(s), n_log_sum
    with context(lattice(model, Lx, Ly, 1.0, h, alpha), n_chains=len(s),
                 solver=vmc.SOLVER_CG) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        out = torch.zeros((len(s), 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, to_dev_spins(s), out)
        got = cplx(out)
    ref = oracle.eloc(model, Lx, Ly, 1.0, h, M, p, s)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= eloc_tolerance(model, Lx, Ly, 1.0, h, M, p, s))


def test_empty_batch_is_a_noop():
    with context(lattice(T, 10, 1, 1.0, 1.0, 1), n_chains=4) as ctx:
        e = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
        s = torch.zeros((0, 10), dtype=torch.int8, device="cuda")
        vmc.vmc_logpsi(ctx, 0, s, e)
        vmc.vmc_local_energy(ctx, 0, s, e)


# (model, Lx, Ly, J, h, alpha, sigma, chains, sweeps)
SAMPLE_CASES = [
    (T, 10, 1, 1.0, 1.0, 1, 0.3, 256, 30),
    (T, 6, 6, 1.0, 3.0, 2, 0.1, 256, 6),
    (H, 8, 8, 1.0, 0.0, 2, 0.05, 512, 4),
    (H, 10, 1, 1.0, 0.0, 1, 0.3, 256, 20),
]


@pytest.mark.parametrize("case", SAMPLE_CASES, ids=["tfim10", "tfim6x6", "heis8x8", "heis10"])
def test_sampler_trajectories_match_oracle(case):
    """Same Philox stream and acceptance rule: every recorded state equals the oracle's,
    except in chains where the oracle met a decision within 1e-4 of the threshold
    (FP32 vs FP64 may decide those differently; then the trajectories part)."""
    model, Lx, Ly, J, h, alpha, sigma, C, sweeps = case
    N, M = Lx * Ly, alpha * Lx * Ly
    p = inputs.rbm_params(N, M, sigma, seed=3, marshall=(Lx, Ly) if model == H else None)
    s0 = inputs.initial_spins(model, C, N, seed=4)
    seed = 12345
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=C, seed=seed,
                 solver=vmc.SOLVER_CG) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s0)
        # two calls: the sweep counter must continue across them
        k1 = sweeps // 2
        out1 = torch.zeros((k1 * C, N), dtype=torch.int8, device="cuda")
        lp1 = torch.zeros((k1 * C, 2), dtype=torch.float32, device="cuda")
        el1 = torch.zeros((k1 * C, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_sample(ctx, 0, 0, k1, out1, lp1, el1)
        out2 = torch.zeros(((sweeps - k1) * C, N), dtype=torch.int8, device="cuda")
        vmc.vmc_sample(ctx, 0, 0, sweeps - k1, out2)
        got = torch.cat([out1, out2]).cpu().numpy().reshape(sweeps, C, N)
        final = vmc.vmc_get_chains(ctx, 0, C, N)
        lp1 = cplx(lp1)
        el1 = cplx(el1)
    fin, rec, margin, acc = oracle.metropolis(model, Lx, Ly, M, p, s0, seed=seed, stream=0,
                                              n_sweeps=sweeps, record=True)
    same = np.all(got == rec, axis=(0, 2))
    assert np.array_equal(final[same], fin[same])
    bad = ~same
    assert np.all(margin[bad] < 1e-4), (np.sum(bad), margin[bad])
    assert bad.mean() <= 0.01
    assert acc.sum() > 0
    if model == H:
        assert np.all(got.sum(axis=2) == 0)
    # fused log psi and E_loc of the recorded samples (first call) against the oracle
    first = got[:k1].reshape(-1, N)
    ref_el = oracle.eloc(model, Lx, Ly, J, h, M, p, first)
    assert np.all(np.abs(el1 - ref_el) <= eloc_tolerance(model, Lx, Ly, J, h, M, p, first))
    if sigma <= 0.05:
        assert np.max(np.abs(el1 - ref_el)) / N <= ELOC_PER_SITE_ABS
    ok = well_conditioned(p, first, N, M)
    assert ok.mean() >= 0.98
    first, lp1 = first[ok], lp1[ok]
    ref_lp = oracle.logpsi(N, M, p, first)
    assert_logpsi_close(lp1, ref_lp, sigma)


def test_sampler_thermalisation_and_sweep_len():
    """n_therm sweeps are run but not recorded; sweep_len overrides N."""
    model, Lx, Ly, alpha, C = T, 8, 1, 1, 64
    N, M = 8, 8
    p = inputs.rbm_params(N, M, 0.2, seed=5)
    s0 = inputs.random_spins(C, N, seed=6)
    with context(lattice(model, Lx, Ly, 1.0, 0.8, alpha), n_chains=C, seed=9, sweep_len=5,
                 solver=vmc.SOLVER_CG) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s0)
        out = torch.zeros((3 * C, N), dtype=torch.int8, device="cuda")
        vmc.vmc_sample(ctx, 0, 4, 3, out)
        got = out.cpu().numpy().reshape(3, C, N)
    _, rec, margin, _ = oracle.metropolis(model, Lx, Ly, M, p, s0, seed=9, n_sweeps=7,
                                          sweep_len=5, record=True)
    same = np.all(got == rec[4:], axis=(0, 2))
    assert np.all(margin[~same] < 1e-4) and same.mean() >= 0.99


# (model, Lx, Ly, J, h, alpha, sigma, n)
GRAD_CASES = [
    (T, 10, 1, 1.0, 1.0, 1, 0.1, 3000),
    (H, 4, 4, 1.0, 0.0, 2, 0.1, 2000),
    (T, 6, 6, 1.0, 3.0, 2, 0.05, 1100),
]


@pytest.mark.parametrize("case", GRAD_CASES, ids=["tfim10", "heis4x4", "tfim6x6"])
def test_grad_and_qfm_match_oracle(case):
    model, Lx, Ly, J, h, alpha, sigma, n = case
    N, M = Lx * Ly, alpha * Lx * Ly
    P = N + M + N * M
    p = inputs.rbm_params(N, M, sigma, seed=41, marshall=(Lx, Ly) if model == H else None)
    s = inputs.initial_spins(model, n, N, seed=42)
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=n, solver=vmc.SOLVER_CHOLESKY_FP64) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        sd = to_dev_spins(s)
        e = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, sd, e)
        O = torch.zeros((n, P, 2), dtype=torch.float32, device="cuda")
        F = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        stats = vmc.vmc_grad(ctx, 0, sd, e, O, F)
        S = torch.zeros((P, P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_qfm(ctx, 0, sd, vmc.PREC_FP32, S)
        E = cplx(e)
        O, F, S = cplx(O), cplx(F), cplx(S)
    Oref = oracle.ok(N, M, p, s)
    assert np.all(np.abs(O - Oref) <= OK_REL * np.abs(Oref) + OK_ABS)
    Sref, Fref, Eref = oracle.sr_matrices(Oref, E)        # same FP32 energies as the GPU used
    assert abs(stats[0] + 1j * stats[1] - Eref) <= 1e-9 * max(1.0, abs(Eref))
    assert np.max(np.abs(F - Fref)) <= F_REL * np.max(np.abs(Fref))
    assert np.max(np.abs(S - Sref)) <= s_tol_fp32(n) * np.max(np.abs(np.diag(Sref)))
    assert np.allclose(S, S.conj().T, atol=0)


@pytest.mark.parametrize("case", GRAD_CASES, ids=["tfim10", "heis4x4", "tfim6x6"])
def test_qfm_bf16split_tensor_cores_match_oracle(case):
    """The tcgen05 BF16-split Gram against the FP64 oracle (ragged 2P against 128-row
    tiles, K not a multiple of the 64-sample stage) and against the FP32 SIMT Gram."""
    model, Lx, Ly, J, h, alpha, sigma, n = case
    N, M = Lx * Ly, alpha * Lx * Ly
    P = N + M + N * M
    p = inputs.rbm_params(N, M, sigma, seed=41, marshall=(Lx, Ly) if model == H else None)
    s = inputs.initial_spins(model, n, N, seed=42)
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=n, solver=vmc.SOLVER_CHOLESKY_MIXED) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        sd = to_dev_spins(s)
        S16 = torch.zeros((P, P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_qfm(ctx, 0, sd, vmc.PREC_BF16SPLIT, S16)
        S32 = torch.zeros((P, P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_qfm(ctx, 0, sd, vmc.PREC_FP32, S32)
        S16, S32 = cplx(S16), cplx(S32)
    Oref = oracle.ok(N, M, p, s)
    Sref, _, _ = oracle.sr_matrices(Oref, np.zeros(n))
    d = np.max(np.abs(np.diag(Sref)))
    assert np.max(np.abs(S16 - Sref)) <= s_tol_bf16(n) * d
    assert np.max(np.abs(S16 - S32)) <= (s_tol_bf16(n) + s_tol_fp32(n)) * d
    assert np.array_equal(S16, S16.conj().T)


@pytest.mark.parametrize("n", [1024, 8192])
def test_qfm_8x8_sampled_entries(n):
    """At the 8x8 Heisenberg benchmark shape (P = 8384, 67 x 67 Gram tiles of 128 rows; at
    n = 8192 the benchmark's sample count, i.e. the timed kernel's full K loop) compare
    sampled entries of S, every F_k and the diagonal with the oracle."""
    model, Lx, Ly, alpha = H, 8, 8, 2
    N, M = 64, 128
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.01, seed=2, marshall=(Lx, Ly))
    s = inputs.random_sz0_spins(n, N, seed=3)
    with context(lattice(model, Lx, Ly, 1.0, 0.0, alpha), n_chains=n, solver=vmc.SOLVER_CHOLESKY_MIXED) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        sd = to_dev_spins(s)
        e = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, sd, e)
        F = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_grad(ctx, 0, sd, e, None, F)
        S = torch.zeros((P, P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_qfm(ctx, 0, sd, vmc.PREC_FP32, S)
        Sd = S.cpu().numpy()
        vmc.vmc_qfm(ctx, 0, sd, vmc.PREC_BF16SPLIT, S)
        Sb = S.cpu().numpy()
        del S
        E, F = cplx(e), cplx(F)
    rng = np.random.default_rng(0)
    kk = np.concatenate([rng.integers(0, P, 300), np.arange(0, P, 97), [P - 1, 0, N, N + M]])
    ll = np.concatenate([rng.integers(0, P, 300), np.arange(0, P, 97)[::-1], [P - 1, P - 1, 3, N + M + 5]])
    O = oracle.ok(N, M, p, s)
    s_ref, f_ref = oracle.sr_entries(O, E, kk, ll, np.arange(P))
    got = Sd[kk, ll, 0] + 1j * Sd[kk, ll, 1]
    gotb = Sb[kk, ll, 0] + 1j * Sb[kk, ll, 1]
    scale = np.max(np.abs(oracle.sr_entries(O, E, np.arange(0, P, 50), np.arange(0, P, 50), [])[0]))
    assert np.max(np.abs(got - s_ref)) <= s_tol_fp32(n) * scale
    assert np.max(np.abs(gotb - s_ref)) <= s_tol_bf16(n) * scale
    assert np.array_equal(Sb[..., 0], Sb[..., 0].T)
    assert np.max(np.abs(F - f_ref)) <= F_REL * np.max(np.abs(f_ref))
    # Hermitian and the Sz = 0 null vector (sum of the a-block columns)
    v = np.zeros(P, np.complex128)
    v[:N] = 1.0
    Sc = Sd[..., 0] + 1j * Sd[..., 1]
    # S v is rounding only; its bound grows with n like the FP32 accumulation bound n 2^-24
    # (1e-5 of the a-block's norm at n = 1024)
    assert np.linalg.norm(Sc @ v) <= 1e-5 * (n / 1024) * np.linalg.norm(Sc[:, :N])
    assert np.array_equal(Sd[..., 0], Sd[..., 0].T) and np.array_equal(Sd[..., 1], -Sd[..., 1].T)


def test_tc_solve_8x8_full_size_residual():
    """The tensor-core solver at the benchmark's size: S (P = 8384) formed by the BF16-split
    Gram from n = 8192 samples, the benchmark's shift 1e-3, vmc_solve with the tensor-core
    Cholesky (17 panels of 512, 131 diagonal blocks, 33 dataflow blocks per triangular
    solve) and refinement.  The returned x must solve the shifted system S~ x = F to a
    relative residual of 1e-10, computed here in FP64 on the host from the same S and F."""
    model, Lx, Ly, alpha, n, nu = H, 8, 8, 2, 8192, 1e-3
    N, M = 64, 128
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.01, seed=1234, marshall=(Lx, Ly))
    s = inputs.random_sz0_spins(n, N, seed=17)
    with context(lattice(model, Lx, Ly, 1.0, 0.0, alpha), n_chains=n, shift=nu,
                 precision=vmc.PREC_BF16SPLIT, solver=vmc.SOLVER_CHOLESKY_TC, cg_tol=1e-10,
                 cg_maxit=50) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        sd = to_dev_spins(s)
        e = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, sd, e)
        F = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_grad(ctx, 0, sd, e, None, F)
        S = torch.zeros((P, P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_qfm(ctx, 0, sd, vmc.PREC_BF16SPLIT, S)
        x = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        it, rel = vmc.vmc_solve(ctx, 0, S, F, x)
        Sh = S.cpu().numpy()
        del S
        F, x = cplx(F), cplx(x)
    Sc = Sh[..., 0] + 1j * Sh[..., 1]
    del Sh
    d = np.real(np.diag(Sc)).copy()
    r = Sc @ x + nu * d * x - F
    res = np.linalg.norm(r) / np.linalg.norm(F)
    assert res <= 1e-10, res
    assert abs(rel - res) <= 0.5 * res + 1e-12
    assert 0 < it <= 50


@pytest.mark.parametrize("solver", [vmc.SOLVER_CHOLESKY_FP64, vmc.SOLVER_CHOLESKY_MIXED,
                                    vmc.SOLVER_CHOLESKY_TC])
@pytest.mark.parametrize("shape", [(T, 10, 1, 1, 1e-4, 0), (H, 4, 4, 2, 1e-3, 0), (T, 6, 6, 1, 1e-2, 1),
                                   (T, 11, 1, 4, 1e-3, 0)],
                         ids=["P120", "P560", "P1332_additive", "P539_odd"])
def test_solve_matches_oracle(solver, shape):
    model, Lx, Ly, alpha, nu, mode = shape
    N, M = Lx * Ly, alpha * Lx * Ly
    P = N + M + N * M
    n = 3 * P
    p = inputs.rbm_params(N, M, 0.1, seed=8, marshall=(Lx, Ly) if model == H else None)
    s = inputs.initial_spins(model, n, N, seed=9)
    O = oracle.ok(N, M, p, s)
    E = oracle.eloc(model, Lx, Ly, 1.0, 1.0, M, p, s)
    S, F, _ = oracle.sr_matrices(O, E)
    xref = oracle.cholesky_solve(oracle.shift(S, nu, mode), F)
    with context(lattice(model, Lx, Ly, 1.0, 1.0, alpha), n_chains=n, solver=solver, shift=nu,
                 shift_mode=mode, cg_tol=1e-12, cg_maxit=60) as ctx:
        Sd = torch.from_numpy(S.view(np.float64).reshape(P, P, 2).copy()).cuda()
        Fd = torch.from_numpy(F.view(np.float64).reshape(P, 2).copy()).cuda()
        xd = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        it, rel = vmc.vmc_solve(ctx, 0, Sd, Fd, xd)
        x = cplx(xd)
    St = oracle.shift(S, nu, mode)
    r = St @ x - F
    res = np.linalg.norm(r) / np.linalg.norm(F)
    sv = np.linalg.svd(St, compute_uv=False)
    cond = sv[0] / sv[-1]
    assert res <= 1e-13 * sv[0] * np.linalg.norm(x) / np.linalg.norm(F) + 1e-14
    assert abs(rel - res) <= 1e-9 + 0.5 * res
    # forward error of any x: |x - x*| <= |St^-1| |St x - F| (x* exact), plus the oracle's
    # own rounding (~1e-16 cond)
    assert np.linalg.norm(x - xref) <= (1.01 * np.linalg.norm(r) / sv[-1]
                                        + 1e-14 * cond * np.linalg.norm(xref) + 1e-12)


def test_solve_reports_non_positive_pivot():
    N, M = 10, 10
    P = N + M + N * M
    with context(lattice(T, 10, 1, 1.0, 1.0, 1), n_chains=4, solver=vmc.SOLVER_CHOLESKY_FP64,
                 shift=0.0) as ctx:
        S = np.eye(P, dtype=np.complex128)
        S[5, 5] = -1.0
        Sd = torch.from_numpy(S.view(np.float64).reshape(P, P, 2).copy()).cuda()
        Fd = torch.ones((P, 2), dtype=torch.float64, device="cuda")
        xd = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        with pytest.raises(vmc.VmcError) as e:
            vmc.vmc_solve(ctx, 0, Sd, Fd, xd)
        assert e.value.status == vmc.VMC_ERR_NUMERIC
        # the context stays usable after the reported failure
        S[5, 5] = 2.0
        Sd = torch.from_numpy(S.view(np.float64).reshape(P, P, 2).copy()).cuda()
        vmc.vmc_solve(ctx, 0, Sd, Fd, xd)


@pytest.mark.parametrize("solver,precision", [(vmc.SOLVER_CHOLESKY_FP64, vmc.PREC_FP32),
                                              (vmc.SOLVER_CHOLESKY_MIXED, vmc.PREC_FP32),
                                              (vmc.SOLVER_CHOLESKY_MIXED, vmc.PREC_BF16SPLIT),
                                              (vmc.SOLVER_CHOLESKY_TC, vmc.PREC_BF16SPLIT),
                                              (vmc.SOLVER_CG, vmc.PREC_FP32),
                                              (vmc.SOLVER_CG, vmc.PREC_BF16SPLIT)])
def test_sr_step_matches_oracle_pipeline(solver, precision):
    """One SR step.  The sample set is read back through vmc_sample on a twin context
    (the kernels are deterministic, and the sampler's agreement with the oracle's
    Metropolis stream is covered above); the oracle then computes E_loc, O_k, S, F, the
    shifted Cholesky solve and the Euler update from it.  The GPU's updated parameters
    must solve the oracle's equation to the accuracy the FP32 S and F allow."""
    model, Lx, Ly, J, h, alpha = T, 10, 1, 1.0, 1.0, 1
    N, M = 10, 10
    C, spc, therm, dt, nu, seed = 64, 20, 5, 0.02, 1e-4, 77
    p = inputs.rbm_params(N, M, 0.01, seed=1234)
    s0 = inputs.random_spins(C, N, seed=99)
    kw = dict(n_chains=C, samples_per_chain=spc, therm_sweeps=therm, seed=seed, solver=solver,
              precision=precision, shift=nu, cg_tol=1e-10, cg_maxit=1000)
    with context(lattice(model, Lx, Ly, J, h, alpha), **kw) as twin:
        vmc.vmc_set_params(twin, 0, p)
        vmc.vmc_set_chains(twin, 0, s0)
        out = torch.zeros((spc * C, N), dtype=torch.int8, device="cuda")
        vmc.vmc_sample(twin, 0, therm, spc, out)
        samples = out.cpu().numpy()
    with context(lattice(model, Lx, Ly, J, h, alpha), **kw) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s0)
        st = vmc.vmc_sr_step(ctx, 0, dt)
        p1 = vmc.vmc_get_params(ctx, 0)
        launches = vmc.vmc_kernel_launches(ctx)
    assert launches > 5
    E = oracle.eloc(model, Lx, Ly, J, h, M, p, samples)
    O = oracle.ok(N, M, p, samples)
    S, F, Em = oracle.sr_matrices(O, E)
    assert abs(st.e_mean_re - Em.real) / N <= ELOC_PER_SITE_ABS
    assert st.n_samples == C * spc
    St = oracle.shift(S, nu, 0)
    delta = (p - p1) / dt
    res = np.linalg.norm(St @ delta - F) / np.linalg.norm(F)
    rel = 1e-4 if precision == vmc.PREC_FP32 else 4e-4
    bound = rel * (1 + np.linalg.norm(St, 2) * np.linalg.norm(delta) / np.linalg.norm(F))
    assert res <= bound, (res, bound)
    assert 0.0 < st.acceptance < 1.0
    assert st.solver_relres <= 1e-10


# --------------------------------------------------------------------------------------
# matrix-free CG (a11)
# --------------------------------------------------------------------------------------
# The CG operator is applied in FP32 (u = Obar v and the F-type reduction with FP32
# sub-sums of 128 samples), so the returned x solves a system within
# CG_OPERATOR_REL * ||S~|| ||x|| of the oracle's FP64 one.
CG_OPERATOR_REL = 128 * 2.0 ** -24 * 8
# On the tensor cores the direction's W block and conj(t) u' are BF16 hi/lo pairs (~2^-17
# relative each, lo.lo dropped: 4 * 2^-16 as for S) and the Obar^H u sums accumulate in FP32
# over K chunks of 2048 samples (worst case 2048 * 2^-24) before the compensated sum of the
# chunks (about one FP32 rounding of the result).
CG_OPERATOR_REL_TC = 4 * 2.0 ** -16 + 2048 * 2.0 ** -24


@pytest.mark.parametrize("precision", [vmc.PREC_FP32, vmc.PREC_BF16SPLIT], ids=["simt", "tc"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape", [(T, 10, 1, 1.0, 1.0, 1, 2000), (H, 4, 4, 1.0, 0.0, 2, 1500),
                                   (T, 6, 6, 1.0, 3.0, 2, 1100)], ids=["tfim10", "heis4x4", "tfim6x6"])
def test_cg_solve_matches_oracle(shape, mode, precision):
    model, Lx, Ly, J, h, alpha, n = shape
    op_rel = CG_OPERATOR_REL if precision == vmc.PREC_FP32 else CG_OPERATOR_REL_TC
    N, M = Lx * Ly, alpha * Lx * Ly
    P = N + M + N * M
    nu = 1e-3 if mode == 0 else 1e-2
    p = inputs.rbm_params(N, M, 0.1, seed=51, marshall=(Lx, Ly) if model == H else None)
    s = inputs.initial_spins(model, n, N, seed=52)
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=n, solver=vmc.SOLVER_CG, shift=nu,
                 shift_mode=mode, cg_tol=1e-8, cg_maxit=2000, precision=precision) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        sd = to_dev_spins(s)
        e = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, sd, e)
        F = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_grad(ctx, 0, sd, e, None, F)
        x = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        it, rel = vmc.vmc_cg_solve(ctx, 0, sd, F, x)
        Fh, xh = cplx(F), cplx(x)
    assert rel <= 1e-8 and 0 < it < 2000
    O = oracle.ok(N, M, p, s)
    S, _, _ = oracle.sr_matrices(O, np.zeros(n))
    St = oracle.shift(S, nu, mode)
    res = np.linalg.norm(St @ xh - Fh) / np.linalg.norm(Fh)
    bound = 1e-8 + op_rel * np.linalg.norm(St, 2) * np.linalg.norm(xh) / np.linalg.norm(Fh)
    assert res <= bound, (res, bound)
    # the oracle's own matrix-free CG reaches the same solution
    xo, ito, relo = oracle.cg_solve(O, Fh, nu, mode, tol=1e-12, maxit=5000)
    assert np.linalg.norm(xh - xo) <= np.linalg.cond(St) * bound * np.linalg.norm(xo)


# (model, Lx, Ly, alpha, n): shapes that exercise every tiling path of the tensor-core
# operator: more 256-sample items than SMs with many K chunks (4x4), N > 128 (two 128-row
# spin tiles, three 64-wide K blocks, three column / row tiles of 128), a ragged sample count
# with three column tiles (8x8), an odd M (unpaired hidden units).
APPLY_SHAPES = [(T, 4, 4, 2, 40000), (T, 130, 1, 1, 1024), (H, 8, 8, 2, 3000), (T, 9, 1, 1, 777)]


@pytest.mark.parametrize("precision", [vmc.PREC_FP32, vmc.PREC_BF16SPLIT], ids=["simt", "tc"])
@pytest.mark.parametrize("shape", APPLY_SHAPES, ids=["items", "n130", "heis8x8", "oddM"])
def test_sr_apply_matches_oracle(shape, precision):
    """One application y = S~ v of the CG operator against the oracle's, entry by entry, on
    samples away from the nodes of psi (|cosh theta_j| >= 0.1).  Bound, to first order:
      the products see each O_qk and v_l with relative error e (BF16 split: 4 * 2^-16;
      FP32: 2^-24) plus FP32 accumulation over at most K terms -> rel * b_k with
      b_k = (1/n) sum_q |O_qk| (sum_l |O_ql| |v_l| + |<O>.v|);
      t = tanh theta is formed in FP32 from an FP32 theta (N + 1 terms), whose rounding
      enters t amplified by 1/|cosh theta|^2 -> dO, propagated through both products."""
    model, Lx, Ly, alpha, n0 = shape
    N, M = Lx * Ly, alpha * Lx * Ly
    P = N + M + N * M
    nu = 1e-3
    p = inputs.rbm_params(N, M, 0.1, seed=61, marshall=(Lx, Ly) if model == H else None)
    s = inputs.initial_spins(model, n0, N, seed=62)
    s = s[well_conditioned(p, s, N, M, cut=0.1)]
    n = len(s)
    assert n >= 0.5 * n0
    rng = np.random.default_rng(63)
    v = rng.normal(size=P) + 1j * rng.normal(size=P)
    with context(lattice(model, Lx, Ly, 1.0, 2.0, alpha), n_chains=n0, solver=vmc.SOLVER_CG,
                 shift=nu, precision=precision) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vd = torch.from_numpy(np.stack([v.real, v.imag], axis=1).copy()).cuda()
        yd = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_sr_apply(ctx, 0, to_dev_spins(s), vd, yd)
        y = cplx(yd)
    O = oracle.ok(N, M, p, s)
    ref = oracle.sr_apply(O, v, nu, 0)
    aO = np.abs(O)
    inner = aO @ np.abs(v) + abs(O.mean(axis=0) @ v)
    rel = (4 * 2.0 ** -16 if precision == vmc.PREC_BF16SPLIT else 2.0 ** -24) \
        + (max(N, M) + 4096) * 2.0 ** -24
    bound = rel * (aO.T @ inner) / n
    # FP32 theta and tanh: |dt_qj| <= (N + 1) 2^-24 (|b_j| + sum_i |W_ji|) / |cosh theta|^2
    #                                 + 4 * 2^-24 |t_qj|
    b, W = p[N:N + M], p[N + M:].reshape(M, N)
    theta = b[None, :] + s.astype(np.float64) @ W.T
    dth = (N + 1) * 2.0 ** -24 * (np.abs(b) + np.abs(W).sum(axis=1))
    dt = dth[None, :] / np.abs(np.cosh(theta)) ** 2 + 4 * 2.0 ** -24 * np.abs(np.tanh(theta))
    dO = np.concatenate([np.zeros((n, N)), dt, np.repeat(dt, N, axis=1)], axis=1)
    du = dO @ np.abs(v)
    bound += (dO.T @ inner + aO.T @ du) / n
    err = np.abs(y - ref)
    assert np.all(err <= bound), (np.max(err / bound), np.argmax(err / bound))
    assert np.linalg.norm(y - ref) <= 1e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [vmc.PREC_FP32, vmc.PREC_BF16SPLIT], ids=["simt", "tc"])
def test_sr_step_cg_heisenberg_16x16(precision):
    """The 16x16 Heisenberg shape (N = 256, M = 512, P = 131 840) through the CG step,
    with fewer chains than the benchmark: the step converges and the energy is physical
    (Pauli units: E/N >= -3, the 2D antiferromagnet's ground state is about -2.68 per site)."""
    Lx = Ly = 16
    N, M = 256, 512
    C = 2048
    p = inputs.rbm_params(N, M, 0.01, seed=1234, marshall=(Lx, Ly))
    with context(lattice(H, Lx, Ly, 1.0, 0.0, 2), n_chains=C, solver=vmc.SOLVER_CG, shift=1e-3,
                 cg_tol=1e-6, cg_maxit=100, therm_sweeps=5, precision=precision) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, inputs.random_sz0_spins(C, N, seed=3))
        st = vmc.vmc_sr_step(ctx, 0, 0.02)
        p1 = vmc.vmc_get_params(ctx, 0)
    assert st.solver_relres <= 1e-6 and st.solver_iters <= 100
    assert -3.0 <= st.e_mean_re / N <= 1.0
    assert np.all(np.isfinite(p1)) and np.linalg.norm(p1 - p) > 0


@pytest.mark.parametrize("precision", [vmc.PREC_FP32, vmc.PREC_BF16SPLIT], ids=["simt", "tc"])
def test_sr_step_cg_16x16_solves_oracle_equation(precision):
    """The CG step at the 16x16 shape (P = 131 840) on a sub-sampled set of 64 chains: the
    samples are read back through a twin context, the oracle forms E_loc, O_k and F, and the
    GPU's update delta = (p - p1) / dt must solve the oracle's shifted equation
    (S + nu diag S) delta = F, applied matrix-free in FP64 (S = Obar^H Obar / n, Eq. qfm),
    to the CG tolerance plus the operator's rounding.  The matrix-free product is first
    checked against the oracle's explicit S on a small slice of the same samples."""
    Lx = Ly = 16
    N, M = 256, 512
    C, therm, dt, nu, seed = 64, 5, 0.02, 1e-3, 21
    p = inputs.rbm_params(N, M, 0.01, seed=1234, marshall=(Lx, Ly))
    s0 = inputs.random_sz0_spins(C, N, seed=3)
    kw = dict(n_chains=C, samples_per_chain=1, therm_sweeps=therm, seed=seed,
              solver=vmc.SOLVER_CG, precision=precision, shift=nu, cg_tol=1e-6, cg_maxit=400)
    with context(lattice(H, Lx, Ly, 1.0, 0.0, 2), **kw) as twin:
        vmc.vmc_set_params(twin, 0, p)
        vmc.vmc_set_chains(twin, 0, s0)
        out = torch.zeros((C, N), dtype=torch.int8, device="cuda")
        vmc.vmc_sample(twin, 0, therm, 1, out)
        samples = out.cpu().numpy()
    with context(lattice(H, Lx, Ly, 1.0, 0.0, 2), **kw) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s0)
        st = vmc.vmc_sr_step(ctx, 0, dt)
        p1 = vmc.vmc_get_params(ctx, 0)
    assert st.solver_relres <= 1e-6 and st.solver_iters <= 400
    E = oracle.eloc(H, Lx, Ly, 1.0, 0.0, M, p, samples)
    O = oracle.ok(N, M, p, samples)
    _, F, Em = oracle.sr_matrices(O, E, want_S=False)
    assert abs(st.e_mean_re - Em.real) / N <= ELOC_PER_SITE_ABS
    Ob = O - O.mean(axis=0)
    dS = np.mean(np.abs(Ob) ** 2, axis=0)

    def s_tilde(v, Obar=Ob, d=dS):
        return Obar.conj().T @ (Obar @ v) / len(Obar) + nu * d * v

    # the matrix-free product against the oracle's explicit S on a slice of parameters
    cols = np.r_[0:40, N:N + 40, N + M:N + M + 80]
    Ssl, _, _ = oracle.sr_matrices(O[:, cols], E)
    v = np.random.default_rng(5).normal(size=len(cols)) + 0j
    Obs = O[:, cols] - O[:, cols].mean(axis=0)
    assert np.allclose(oracle.shift(Ssl, nu, 0) @ v,
                       s_tilde(v, Obs, np.mean(np.abs(Obs) ** 2, axis=0)), rtol=1e-12, atol=1e-14)
    delta = (p - p1) / dt
    res = np.linalg.norm(s_tilde(delta) - F) / np.linalg.norm(F)
    # |S~|_2 <= |Obar|_2^2 / n + nu max diag S (the Gram of the n x n side is small)
    norm_s = np.linalg.eigvalsh(Ob @ Ob.conj().T / C).max() + nu * dS.max()
    op = CG_OPERATOR_REL if precision == vmc.PREC_FP32 else CG_OPERATOR_REL_TC
    bound = 2e-6 + op * (1 + norm_s * np.linalg.norm(delta) / np.linalg.norm(F))
    assert res <= bound, (res, bound)


def test_sr_step_bf16_split_recovers_from_indefinite_s():
    """1D TFIM N = 10 near the uniform state with a 1e-4 relative shift: the three-product
    BF16 split can make the shifted S indefinite (its error is minus the PSD lo.lo^T term);
    the step then re-forms S with the fourth product and solves.  (The two updates are not
    compared entry by entry: S~ has a condition number near 1e8 here, so the FP32 and BF16
    roundings of S move the solution far along its near-null directions.)"""
    N, M, C, spc = 10, 10, 256, 200
    p = inputs.rbm_params(N, M, 0.01, seed=1234)
    s0 = inputs.random_spins(C, N, seed=99)
    out = {}
    for prec in (vmc.PREC_FP32, vmc.PREC_BF16SPLIT):
        with context(lattice(T, N, 1, 1.0, 1.0, 1), n_chains=C, samples_per_chain=spc,
                     solver=vmc.SOLVER_CHOLESKY_MIXED, shift=1e-4, precision=prec, seed=1) as ctx:
            vmc.vmc_set_params(ctx, 0, p)
            vmc.vmc_set_chains(ctx, 0, s0)
            st = vmc.vmc_sr_step(ctx, 0, 0.02)
            out[prec] = (st, vmc.vmc_get_params(ctx, 0))
    for prec, (st, p1) in out.items():
        assert st.solver_relres <= 1e-10 and np.all(np.isfinite(p1))
    # same samples (same seed, same sampler), so the energies agree exactly
    assert out[vmc.PREC_FP32][0].e_mean_re == out[vmc.PREC_BF16SPLIT][0].e_mean_re
    for prec in out:
        assert np.linalg.norm(out[prec][1] - p) > 0


def test_cfg1_sampled_sr_reaches_jordan_wigner_energy():
    """The sampled GPU SR loop of the 1D TFIM workload (N = 10, J = h = 1, alpha = 1, 256
    chains x 200 samples, dt 0.02, shift 1e-4, plain FP32 path) drives the RBM to within
    1e-3 (relative) of the Jordan-Wigner ground energy E0 = -12.784906443 (section "Ground
    state search": the fermionised chain is the exact reference).  The energy judged is the
    exact variational energy of the GPU's parameters (oracle enumeration of all 1024
    states), checked every 25 steps, at most 2000 steps."""
    N, M, J, h = 10, 10, 1.0, 1.0
    k = (2 * np.arange(N) + 1) * np.pi / N
    E0 = -np.sum(np.sqrt(J * J + h * h - 2 * J * h * np.cos(k)))
    assert abs(E0 + 12.784906443) < 1e-8
    p = inputs.rbm_params(N, M, 0.01, seed=1234)
    with context(lattice(T, N, 1, J, h, 1), n_chains=256, samples_per_chain=200,
                 therm_sweeps=20, seed=1, solver=vmc.SOLVER_CHOLESKY_MIXED, shift=1e-4,
                 precision=vmc.PREC_FP32, cg_tol=1e-10, cg_maxit=50) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, inputs.random_spins(256, N, seed=99))
        hist = []
        for step in range(1, 2001):
            st = vmc.vmc_sr_step(ctx, 0, 0.02)
            hist.append(st.e_mean_re)
            if step % 25 == 0:
                pk = vmc.vmc_get_params(ctx, 0)
                e_exact = oracle.exact_energy(T, N, 1, J, h, M, pk)[0].real
                if abs(e_exact - E0) / abs(E0) <= 1e-3:
                    break
    assert abs(e_exact - E0) / abs(E0) <= 1e-3, (step, e_exact, E0)
    # the sampled estimate of the last steps agrees with the exact energy
    assert abs(np.mean(hist[-10:]) - e_exact) <= 0.01 * abs(E0)


def test_cg_non_convergence_is_reported():
    """A CG that stops at cg_maxit above cg_tol is an error (VMC_ERR_NUMERIC), both from
    vmc_cg_solve (x holds the last iterate) and from vmc_sr_step (the parameters are left
    unchanged and the statistics say solver_converged = 0); the context keeps working."""
    N, M, C = 10, 10, 512
    p = inputs.rbm_params(N, M, 0.1, seed=51)
    s = inputs.random_spins(C, N, seed=52)
    P = N + M + N * M
    with context(lattice(T, N, 1, 1.0, 1.0, 1), n_chains=C, solver=vmc.SOLVER_CG, shift=1e-4,
                 cg_tol=1e-14, cg_maxit=2, therm_sweeps=2) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s)
        sd = to_dev_spins(s)
        e = torch.zeros((C, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, sd, e)
        F = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        vmc.vmc_grad(ctx, 0, sd, e, None, F)
        x = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        with pytest.raises(vmc.VmcError) as ei:
            vmc.vmc_cg_solve(ctx, 0, sd, F, x)
        assert ei.value.status == vmc.VMC_ERR_NUMERIC
        assert ei.value.iters == 2 and ei.value.relres > 1e-14
        assert np.all(np.isfinite(x.cpu().numpy())) and torch.any(x != 0)
        with pytest.raises(vmc.VmcError) as ei:
            vmc.vmc_sr_step(ctx, 0, 0.02)
        assert ei.value.status == vmc.VMC_ERR_NUMERIC
        st = ei.value.stats
        assert st.solver_converged == 0 and st.solver_iters == 2 and st.solver_relres > 1e-14
        assert np.isfinite(st.e_mean_re)
        assert np.array_equal(vmc.vmc_get_params(ctx, 0), p)
        out = torch.zeros((C, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_logpsi(ctx, 0, sd, out)
        assert np.all(np.isfinite(out.cpu().numpy()))


@pytest.mark.parametrize("solver,precision", [(vmc.SOLVER_CHOLESKY_MIXED, vmc.PREC_FP32),
                                              (vmc.SOLVER_CHOLESKY_TC, vmc.PREC_BF16SPLIT)],
                         ids=["fp32_mixed", "tc"])
def test_sr_step_on_given_samples_solves_oracle_equation(solver, precision):
    """vmc_sr_step_on: the SR step on a caller's sample set.  6x6 TFIM with alpha = 2 (P =
    2700: six 512-column panels of the tensor-core factorisation, whose S is one FP16
    product preconditioning CG on the exact FP32 operator); the oracle forms E_loc, O_k, S
    and F from the very same configurations, and the GPU's update must solve the oracle's
    shifted equation (Eq. qfm, the diagonal shift) as in the sampled SR step.  The chains
    do not move, and a sample count other than n_chains * samples_per_chain is refused."""
    model, Lx, Ly, J, h, alpha = T, 6, 6, 1.0, 3.0, 2
    N, M = Lx * Ly, alpha * Lx * Ly
    C, spc, dt, nu = 256, 8, 0.02, 1e-3
    p = inputs.rbm_params(N, M, 0.05, seed=1234)
    s0 = inputs.random_spins(C, N, seed=98)
    samples = inputs.random_spins(C * spc, N, seed=97)
    with context(lattice(model, Lx, Ly, J, h, alpha), n_chains=C, samples_per_chain=spc,
                 therm_sweeps=2, seed=5, solver=solver, precision=precision, shift=nu,
                 cg_tol=1e-8, cg_maxit=200) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s0)
        sd = to_dev_spins(samples)
        with pytest.raises(vmc.VmcError) as ei:
            vmc.vmc_sr_step_on(ctx, 0, sd[:-1], dt)
        assert ei.value.status == vmc.VMC_ERR_ARG
        st = vmc.vmc_sr_step_on(ctx, 0, sd, dt)
        p1 = vmc.vmc_get_params(ctx, 0)
        assert np.array_equal(vmc.vmc_get_chains(ctx, 0, C, N), s0)
    E = oracle.eloc(model, Lx, Ly, J, h, M, p, samples)
    O = oracle.ok(N, M, p, samples)
    S, F, Em = oracle.sr_matrices(O, E)
    assert abs(st.e_mean_re - Em.real) / N <= ELOC_PER_SITE_ABS
    assert st.n_samples == C * spc and st.acceptance == 0.0
    assert st.solver_converged == 1 and st.solver_relres <= 1e-8
    if solver == vmc.SOLVER_CHOLESKY_TC:
        # the factor of the FP16 Gram is a near-exact preconditioner: a wrong factor input
        # would show as a long CG, not as a wrong answer
        assert st.solver_iters <= 25, st.solver_iters
    St = oracle.shift(S, nu, 0)
    delta = (p - p1) / dt
    res = np.linalg.norm(St @ delta - F) / np.linalg.norm(F)
    bound = 1e-4 * (1 + np.linalg.norm(St, 2) * np.linalg.norm(delta) / np.linalg.norm(F))
    assert res <= bound, (res, bound)
