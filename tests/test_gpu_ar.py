"""GPU parity of the autoregressive network used as the ansatz (vmc_ar_*) with the FP64
oracle (oracle/ar.py): log psi, exact draws, local energies, log-derivatives and F, one SR
step, independence of the draws, and SR reaching the Jordan-Wigner energy."""
import numpy as np
import pytest

import oracle
from oracle import ar
from paper_2108_03409_b300 import inputs, vmc

from gpu_helpers import cplx, to_dev_spins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T, HEIS = inputs.MODEL_TFIM, inputs.MODEL_HEIS
U24 = 2.0 ** -24


def _ctx(model, Lx, Ly, J, h, H, C, spc=1, seed=11, solver=vmc.SOLVER_CHOLESKY_FP64, shift=1e-3,
         mode=1):
    cfg = vmc.make_config(seed=seed, n_chains=C, samples_per_chain=spc, solver=solver, shift=shift,
                          shift_mode=mode, made_hidden=H, ar_ansatz=1, cg_tol=1e-10, cg_maxit=50)
    return vmc.vmc_init(cfg, [vmc.make_lattice(model, Lx, Ly, J, h, 1)])


def _params(N, H, seed, scale=1.0):
    return inputs.made_params(N, H, seed=seed, scale=scale).astype(np.float64)


def test_ar_logpsi_and_draws_match_oracle():
    """log psi = (1/2) log q against the oracle (FP32 forward: 1e-6 N + 1e-6 |log q|), and
    the exact draws follow the oracle's Philox stream (same round counter) except where the
    oracle met a uniform within 1e-5 of sigma(z)."""
    N, H, n = 10, 32, 2048
    p = _params(N, H, 3, 1.3)
    ctx = _ctx(T, N, 1, 1.0, 1.0, H, n)
    try:
        vmc.vmc_ar_set_params(ctx, 0, p)
        assert np.array_equal(vmc.vmc_ar_get_params(ctx, 0, p.size), p)
        s = inputs.random_spins(n, N, seed=4)
        lp = torch.zeros(n, dtype=torch.float32, device="cuda")
        vmc.vmc_ar_logpsi(ctx, 0, to_dev_spins(s), lp)
        got = lp.cpu().numpy().astype(np.float64)
        sd = torch.zeros((n, N), dtype=torch.int8, device="cuda")
        ld = torch.zeros(n, dtype=torch.float32, device="cuda")
        vmc.vmc_ar_sample(ctx, 0, sd, ld)               # round 0
        draws = sd.cpu().numpy()
        ldraw = ld.cpu().numpy().astype(np.float64)
    finally:
        vmc.vmc_destroy(ctx)
    ref = ar.ar_logpsi(N, H, p, s)
    assert np.all(np.abs(got - ref) <= 0.5 * (2e-6 * N + 1e-6 * np.abs(2 * ref)))
    sref, lqref, margin = oracle.made_sample(N, H, p, n, seed=11, stream=0, round_=0)
    same = np.all(draws == sref, axis=1)
    assert np.all(margin[~same] < 1e-5) and same.mean() >= 0.99
    assert np.all(np.abs(ldraw[same] - 0.5 * lqref[same]) <= 0.5 * (2e-6 * N + 1e-6 * np.abs(lqref[same])))


@pytest.mark.parametrize("model,Lx,Ly,J,h", [(T, 10, 1, 1.0, 0.8), (HEIS, 4, 2, 1.0, 0.0)],
                         ids=["tfim10", "heis4x2"])
def test_ar_local_energy_matches_oracle(model, Lx, Ly, J, h):
    """E_loc(s) = sum_s' H_ss' (q(s')/q(s))^(1/2): each ratio from two FP32 forward passes
    (|d log q| <= 2e-6 N + 1e-6 |log q| each), so |dE| <= sum |H_ss' ratio| * that + 1e-6 |E|."""
    N, H, n = Lx * Ly, 32, 1000
    p = _params(N, H, 5, 1.2)
    s = inputs.random_spins(n, N, seed=6)
    ctx = _ctx(model, Lx, Ly, J, h, H, n)
    try:
        vmc.vmc_ar_set_params(ctx, 0, p)
        e = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_ar_local_energy(ctx, 0, to_dev_spins(s), e)
        got = cplx(e)
    finally:
        vmc.vmc_destroy(ctx)
    ref = ar.ar_eloc(model, Lx, Ly, J, h, H, p, s)
    lq = oracle.made_forward(N, H, p, s)
    scale = np.zeros(n)
    for q in range(n):
        sp, el = oracle.connected(model, Lx, Ly, J, h, s[q])
        lqs = oracle.made_forward(N, H, p, sp)
        scale[q] = np.sum(np.abs(el[1:]) * np.exp(0.5 * (lqs[1:] - lqs[0])))
    tol = scale * (2e-6 * N + 1e-6 * (np.abs(lq) + 10)) + 1e-6 * np.abs(ref) + 1e-6 * N
    assert np.all(np.abs(got.real - ref) <= tol)
    assert np.all(got.imag == 0)


def test_ar_grad_matches_oracle():
    """Per-sample O_k = (1/2) d log q / d theta_k (relative 1e-5 of the largest |O| per
    sample; masked entries exactly 0), <O> and F = <O (E - <E>)> (FP64 sums of FP32 terms:
    1e-5 of max |F|)."""
    N, H, n = 8, 32, 600
    P = oracle.made_nparams(N, H)
    p = _params(N, H, 7, 1.2)
    s = inputs.random_spins(n, N, seed=8)
    ctx = _ctx(T, N, 1, 1.0, 1.0, H, n)
    try:
        vmc.vmc_ar_set_params(ctx, 0, p)
        sd = to_dev_spins(s)
        e = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_ar_local_energy(ctx, 0, sd, e)
        O = torch.zeros((n, P), dtype=torch.float32, device="cuda")
        mo = torch.zeros(P, dtype=torch.float64, device="cuda")
        F = torch.zeros(P, dtype=torch.float64, device="cuda")
        es = vmc.vmc_ar_grad(ctx, 0, sd, e, O, mo, F)
        O, mo, F = (t.cpu().numpy().astype(np.float64) for t in (O, mo, F))
        E = e[:, 0].cpu().numpy().astype(np.float64)
    finally:
        vmc.vmc_destroy(ctx)
    Oref = ar.ar_ok(N, H, p, s)
    big = np.max(np.abs(Oref), axis=1, keepdims=True)
    assert np.all(np.abs(O - Oref) <= 1e-5 * big + 1e-7)
    assert np.all(O[Oref == 0.0] == 0.0)
    _, Fref, Em = oracle.sr_matrices(Oref, E)
    assert abs(es[0] - Em.real) <= 1e-9 * abs(Em)
    assert np.max(np.abs(mo - Oref.mean(axis=0))) <= 1e-5 * np.max(np.abs(Oref))
    assert np.max(np.abs(F - Fref.real)) <= 1e-5 * np.max(np.abs(Fref))


def test_ar_sr_step_matches_oracle_pipeline():
    """One SR step: the draws are reproduced by vmc_ar_sample on a twin context (same seed
    and round counter); the oracle forms E_loc, O, S, F, the additively shifted solve and
    the update from them, and the GPU's update must solve the oracle's equation to the
    accuracy the FP32 S and F allow."""
    N, H, C, spc, dt, nu = 8, 32, 128, 16, 0.05, 1e-3
    Ns = C * spc
    p = _params(N, H, 9)
    twin = _ctx(T, N, 1, 1.0, 1.0, H, C, spc)
    try:
        vmc.vmc_ar_set_params(twin, 0, p)
        sd = torch.zeros((Ns, N), dtype=torch.int8, device="cuda")
        vmc.vmc_ar_sample(twin, 0, sd)
        samples = sd.cpu().numpy()
    finally:
        vmc.vmc_destroy(twin)
    ctx = _ctx(T, N, 1, 1.0, 1.0, H, C, spc)
    try:
        vmc.vmc_ar_set_params(ctx, 0, p)
        st = vmc.vmc_ar_sr_step(ctx, 0, dt)
        p1 = vmc.vmc_ar_get_params(ctx, 0, p.size)
    finally:
        vmc.vmc_destroy(ctx)
    E = ar.ar_eloc(T, N, 1, 1.0, 1.0, H, p, samples)
    O = ar.ar_ok(N, H, p, samples)
    S, F, Em = oracle.sr_matrices(O, E)
    S, F = S.real, F.real
    frozen = np.diag(S) == 0
    St = S + nu * np.eye(len(F))
    St[frozen, frozen] = 1.0 + nu
    delta = (p - p1) / dt
    assert np.all(delta[frozen] == 0)
    res = np.linalg.norm(St @ delta - F) / np.linalg.norm(F)
    bound = 1e-4 * (1 + np.linalg.norm(St, 2) * np.linalg.norm(delta) / np.linalg.norm(F))
    assert res <= bound, (res, bound)
    assert abs(st.e_mean_re - Em.real) <= 1e-5 * N
    assert st.acceptance == 1.0 and st.n_samples == Ns


def test_ar_draws_are_independent():
    """Direct sampling has no Markov chain: consecutive draws are independent, so the pooled
    autocorrelation of the local-energy series at lags 1 and 2 vanishes (its standard error
    is 1/sqrt(C R) = 0.0055 here; bound 0.025) and tau_int = 1/2 + sum_t rho(t) is 1/2."""
    N, H, C, R = 10, 32, 512, 64
    p = _params(N, H, 13, 1.5)
    ctx = _ctx(T, N, 1, 1.0, 1.0, H, C)
    try:
        vmc.vmc_ar_set_params(ctx, 0, p)
        series = []
        sd = torch.zeros((C, N), dtype=torch.int8, device="cuda")
        e = torch.zeros((C, 2), dtype=torch.float32, device="cuda")
        for _ in range(R):
            vmc.vmc_ar_sample(ctx, 0, sd)
            vmc.vmc_ar_local_energy(ctx, 0, sd, e)
            series.append(e[:, 0].double().cpu().numpy())
    finally:
        vmc.vmc_destroy(ctx)
    x = np.array(series)                      # [R][C], every entry an independent draw
    d = x - x.mean()                          # (a per-column mean would bias rho(t) by -1/R)
    var = np.sum(d * d)
    for lag in (1, 2):
        rho = np.sum(d[:-lag] * d[lag:]) / var
        assert abs(rho) <= 0.025, (lag, rho)
    tau = 0.5 + sum(np.sum(d[:-t] * d[t:]) / var for t in (1, 2, 3))
    assert abs(tau - 0.5) <= 0.04, tau


def test_ar_sr_reaches_jordan_wigner():
    """SR of the autoregressive ansatz on the GPU (N = 10 chain, J = h = 1, H = 32, 256 x 200
    direct draws per step, dt 0.05, additive shift 1e-3) reaches 2e-3 of the Jordan-Wigner
    energy (exact energy of the GPU's parameters, checked every 25 steps, at most 400)."""
    N, H, J, h = 10, 32, 1.0, 1.0
    k = (2 * np.arange(N) + 1) * np.pi / N
    E0 = -np.sum(np.sqrt(J * J + h * h - 2 * J * h * np.cos(k)))
    p = _params(N, H, 5)
    ctx = _ctx(T, N, 1, J, h, H, 256, 200, solver=vmc.SOLVER_CHOLESKY_MIXED)
    try:
        vmc.vmc_ar_set_params(ctx, 0, p)
        for step in range(1, 401):
            vmc.vmc_ar_sr_step(ctx, 0, 0.05)
            if step % 25 == 0:
                e_exact = ar.ar_exact_energy(T, N, 1, J, h, H, vmc.vmc_ar_get_params(ctx, 0, p.size))[0]
                if abs(e_exact - E0) / abs(E0) <= 2e-3:
                    break
    finally:
        vmc.vmc_destroy(ctx)
    assert abs(e_exact - E0) / abs(E0) <= 2e-3, (step, e_exact, E0)
