"""GPU parity of the translation-symmetric CNN-ELU ansatz (vmc_cnn_*) with the FP64 oracle
(oracle/cnn.py): log psi, E_loc, log-derivatives, Metropolis trajectories on the shared
Philox stream, one ground-state step, and the paper's recipe reaching the Jordan-Wigner
energy."""
import numpy as np
import pytest

import oracle
from oracle import cnn, tdvp
from paper_2108_03409_b300 import inputs, vmc

from gpu_helpers import cplx, to_dev_spins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T = inputs.MODEL_TFIM
U24 = 2.0 ** -24


def _ctx(N, alpha, h, C, spc=1, seed=21, therm=20):
    cfg = vmc.make_config(seed=seed, n_chains=C, samples_per_chain=spc, therm_sweeps=therm,
                          solver=vmc.SOLVER_CG, tdvp=1, cnn_ansatz=1)
    return vmc.vmc_init(cfg, [vmc.make_lattice(T, N, 1, 1.0, h, alpha)])


def _params(N, alpha, seed, sigma=0.3):
    return np.random.default_rng(seed).normal(0.0, sigma, cnn.nparams(N, alpha))


def _dz_bound(N, alpha, p):
    """FP32 error of every pre-activation: (N + 1) 2^-24 (|b_a| + sum_l |W_al|), summed over
    the alpha N terms of log psi (|f'| <= max(1, e^z) <= 1 + |z| covered by the factor 2)."""
    W = p[:alpha * N].reshape(alpha, N)
    b = p[alpha * N:]
    per = (N + 1) * U24 * (np.abs(b) + np.abs(W).sum(axis=1))
    return 2 * N * per.sum() + 4 * alpha * N * U24


@pytest.mark.parametrize("N,alpha", [(10, 2), (20, 4)])
def test_cnn_eval_matches_oracle(N, alpha):
    n, h = 500, 0.7
    p = _params(N, alpha, 1)
    s = inputs.random_spins(n, N, seed=2)
    ctx = _ctx(N, alpha, h, n)
    try:
        vmc.vmc_cnn_set_params(ctx, 0, p)
        assert np.array_equal(vmc.vmc_cnn_get_params(ctx, 0, p.size), p)
        lp = torch.zeros(n, dtype=torch.float32, device="cuda")
        el = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_cnn_eval(ctx, 0, to_dev_spins(s), lp, el)
        lp = lp.cpu().numpy().astype(np.float64)
        el = cplx(el)
    finally:
        vmc.vmc_destroy(ctx)
    ref = cnn.logpsi(N, alpha, p, s)
    db = _dz_bound(N, alpha, p)
    assert np.all(np.abs(lp - ref) <= db + 4 * U24 * np.abs(ref)), np.max(np.abs(lp - ref)) / db
    eref = cnn.eloc(T, N, 1, 1.0, h, alpha, p, s)
    # each ratio exp(delta) carries twice the log psi bound (delta from the cached z)
    ratios = np.zeros(n)
    for q in range(n):
        sp, e = oracle.connected(T, N, 1, 1.0, h, s[q])
        l = cnn.logpsi(N, alpha, p, sp)
        ratios[q] = np.sum(np.abs(e[1:]) * np.exp(l[1:] - l[0]))
    tol = ratios * (2 * db + 1e-6) + 1e-5 * N
    assert np.all(np.abs(el.real - eref) <= tol)
    assert np.all(el.imag == 0)


def test_cnn_log_derivatives_match_oracle():
    N, alpha, n = 12, 3, 400
    P = cnn.nparams(N, alpha)
    p = _params(N, alpha, 3)
    s = inputs.random_spins(n, N, seed=4)
    ctx = _ctx(N, alpha, 1.0, n)
    try:
        vmc.vmc_cnn_set_params(ctx, 0, p)
        O = torch.zeros((n, P), dtype=torch.float32, device="cuda")
        vmc.vmc_cnn_grad(ctx, 0, to_dev_spins(s), O)
        O = O.cpu().numpy().astype(np.float64)
    finally:
        vmc.vmc_destroy(ctx)
    ref = cnn.ok(N, alpha, p, s)
    assert np.all(np.abs(O - ref) <= 1e-5 * np.max(np.abs(ref), axis=1, keepdims=True) + 1e-6)


def test_cnn_sampler_trajectories_match_oracle():
    """Same Philox stream and acceptance rule: every recorded state equals the oracle's
    Metropolis chain, except in chains whose oracle margin fell below 1e-4."""
    N, alpha, C, sweeps, seed = 10, 2, 128, 6, 33
    p = _params(N, alpha, 5, sigma=0.4)
    s0 = inputs.random_spins(C, N, seed=6)
    ctx = _ctx(N, alpha, 0.9, C, seed=seed)
    try:
        vmc.vmc_cnn_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s0)
        out = torch.zeros((sweeps * C, N), dtype=torch.int8, device="cuda")
        lp = torch.zeros(sweeps * C, dtype=torch.float32, device="cuda")
        vmc.vmc_cnn_sample(ctx, 0, 0, sweeps, out, lp)
        got = out.cpu().numpy().reshape(sweeps, C, N)
        lp = lp.cpu().numpy().astype(np.float64).reshape(sweeps, C)
    finally:
        vmc.vmc_destroy(ctx)
    fin, rec, margin = cnn.metropolis(N, alpha, p, s0, seed=seed, n_sweeps=sweeps, record=True)
    same = np.all(got == rec, axis=(0, 2))
    assert np.all(margin[~same] < 1e-4) and same.mean() >= 0.97, np.sum(~same)
    ref = cnn.logpsi(N, alpha, p, got.reshape(-1, N)).reshape(sweeps, C)
    assert np.max(np.abs(lp - ref)) <= _dz_bound(N, alpha, p) + 4 * U24 * np.max(np.abs(ref))


def test_cnn_ground_state_step_matches_oracle():
    """One step of the recipe (shift nu = 10, pseudo-inverse cutoff 1e-8, tau = 1e-2) on the
    GPU's own samples (reproduced by a twin context with the same stream): the oracle's
    thetadot from the same configurations, within the FP32-input bound amplified by the
    condition number of the shifted S."""
    N, alpha, C, spc, nu, dt = 10, 2, 64, 32, 10.0, 1e-2
    P = cnn.nparams(N, alpha)
    p = _params(N, alpha, 7, sigma=0.1)
    s0 = inputs.random_spins(C, N, seed=8)
    opts = vmc.make_tdvp_opts(gamma=1.0, shift=nu, eps_pinv=1e-8)
    twin = _ctx(N, alpha, 0.7, C, spc)
    try:
        vmc.vmc_cnn_set_params(twin, 0, p)
        vmc.vmc_set_chains(twin, 0, s0)
        sp = torch.zeros((C * spc, N), dtype=torch.int8, device="cuda")
        vmc.vmc_cnn_sample(twin, 0, 20, spc, sp)
        samples = sp.cpu().numpy()
    finally:
        vmc.vmc_destroy(twin)
    ctx = _ctx(N, alpha, 0.7, C, spc)
    try:
        vmc.vmc_cnn_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s0)
        st = vmc.vmc_cnn_sr_step(ctx, 0, dt, opts)
        p1 = vmc.vmc_cnn_get_params(ctx, 0, P)
    finally:
        vmc.vmc_destroy(ctx)
    O = cnn.ok(N, alpha, p, samples)
    E = cnn.eloc(T, N, 1, 1.0, 0.7, alpha, p, samples)
    td, info = tdvp.tdvp_rhs(O, E, gamma=1.0, eps_pinv=1e-8, soft=True, shift=nu)
    ref = p + dt * td.real
    cond = np.max(info["lam"]) / np.min(info["lam"])
    assert np.linalg.norm(p1 - ref) <= 40 * (N + 1) * U24 * cond * dt * np.linalg.norm(td)
    assert abs(st.e_mean_re - info["E"].real) <= 1e-5 * N


def test_cnn_ground_state_recipe_reaches_jordan_wigner():
    """The paper's example on the GPU: L = 10, g = 0.7, alpha = 2, N_MC = 4e4 (200 chains x
    200 samples), tau = 1e-2, nu = 10 * 0.95^n, eps_pinv = 1e-8: the exact energy of the
    GPU's parameters (oracle enumeration, every 25 steps, at most 400) comes within 2e-3 of
    the Jordan-Wigner energy."""
    N, alpha, J, g = 10, 2, 1.0, 0.7
    k = (2 * np.arange(N) + 1) * np.pi / N
    E0 = -np.sum(np.sqrt(J * J + g * g - 2 * J * g * np.cos(k)))
    P = cnn.nparams(N, alpha)
    p = np.random.default_rng(1).normal(0, 0.1, P)
    states = oracle.all_states(N)
    ctx = _ctx(N, alpha, g, 200, 200)
    try:
        vmc.vmc_cnn_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, inputs.random_spins(200, N, seed=9))
        for n in range(400):
            opts = vmc.make_tdvp_opts(gamma=1.0, shift=10.0 * 0.95 ** n, eps_pinv=1e-8)
            st = vmc.vmc_cnn_sr_step(ctx, 0, 1e-2, opts)
            if (n + 1) % 25 == 0:
                q = vmc.vmc_cnn_get_params(ctx, 0, P)
                lp = cnn.logpsi(N, alpha, q, states)
                w = np.exp(2 * (lp - lp.max()))
                e_exact = np.sum(w * cnn.eloc(T, N, 1, J, g, alpha, q, states)) / w.sum()
                if abs(e_exact - E0) / abs(E0) <= 2e-3:
                    break
    finally:
        vmc.vmc_destroy(ctx)
    assert abs(e_exact - E0) / abs(E0) <= 2e-3, (n, e_exact, E0)
