"""GPU parity of the excited-state search by projection (vmc_excited_lambda,
vmc_excited_rhs, vmc_excited_step) with the FP64 oracle (oracle/excited.py), and the search
reaching the first excited energy of exact diagonalisation."""
import numpy as np
import pytest

import oracle
from oracle import excited
from paper_2108_03409_b300 import inputs, vmc

from gpu_helpers import cplx, to_dev_spins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T = inputs.MODEL_TFIM
U24 = 2.0 ** -24


def _ctx(N, J, h, C, spc=1):
    lat = vmc.make_lattice(T, N, 1, J, h, 1)
    cfg = vmc.make_config(seed=3, n_chains=C, samples_per_chain=spc, therm_sweeps=20,
                          solver=vmc.SOLVER_CG, tdvp=1)
    return vmc.vmc_init(cfg, [lat, lat])


def _ground_state(N, M, J, h, steps):
    p = inputs.rbm_params(N, M, 0.01, seed=1234)
    for _ in range(steps):
        S, F, E = oracle.exact_sr(T, N, 1, J, h, M, p)
        p = oracle.update(p, oracle.cholesky_solve(oracle.shift(S, 1e-4, 0), F), 0.05)
    return p


def _e_levels(N, J, h):
    from test_oracle_pins import _dense_h
    return np.linalg.eigvalsh(_dense_h(T, N, 1, J, h).toarray())


def test_lambda_matches_oracle():
    """lambda = <psi/phi> from the same samples (mean of exp(log psi - log phi) with FP32 log
    amplitudes: relative 1e-5), and with exact sums over all states."""
    N, M, n = 8, 8, 2000
    p_psi = inputs.rbm_params(N, M, 0.3, seed=5)
    p_phi = inputs.rbm_params(N, M, 0.3, seed=6)
    s = inputs.random_spins(n, N, seed=7)
    ctx = _ctx(N, 1.0, 0.8, n)
    try:
        vmc.vmc_set_params(ctx, 0, p_psi)
        vmc.vmc_set_params(ctx, 1, p_phi)
        got = vmc.vmc_excited_lambda(ctx, 0, 1, to_dev_spins(s))
        got_ex = vmc.vmc_excited_lambda(ctx, 0, 1, None, exact=1)
    finally:
        vmc.vmc_destroy(ctx)
    ref = excited.overlap_ratio(N, M, p_psi, p_phi, s)
    ref_ex = excited.overlap_ratio_exact(N, M, p_psi, p_phi)
    assert abs(got - ref) <= 1e-5 * abs(ref)
    assert abs(got_ex - ref_ex) <= 1e-5 * abs(ref_ex)


def test_excited_rhs_matches_oracle():
    """The SR direction of Psi = psi - lambda phi on given samples of |psi|^2 and a given
    lambda: importance weights, E_loc^Psi, O^Psi and the FP64 core against the oracle, to
    the FP32-input bound 40 (N + 1) 2^-24 / eps_pinv (soft cutoff), and <E>_Psi to 1e-5."""
    N, M, n, eps = 8, 8, 3000, 1e-3
    P = N + M + N * M
    p_psi = inputs.rbm_params(N, M, 0.3, seed=15)
    p_phi = inputs.rbm_params(N, M, 0.3, seed=16)
    s = inputs.random_spins(n, N, seed=17)
    lam = 0.4 - 0.25j
    opts = vmc.make_tdvp_opts(gamma=1.0, eps_pinv=eps, shift=1e-3)
    ctx = _ctx(N, 1.0, 0.8, n)
    try:
        vmc.vmc_set_params(ctx, 0, p_psi)
        vmc.vmc_set_params(ctx, 1, p_phi)
        out = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
        st = vmc.vmc_excited_rhs(ctx, 0, 1, opts, out, spins_psi=to_dev_spins(s), lam=lam)
        got = cplx(out)
    finally:
        vmc.vmc_destroy(ctx)
    ref, info = excited.excited_rhs(T, N, 1, 1.0, 0.8, M, p_psi, p_phi, lam, s, shift=1e-3,
                                    eps_pinv=eps)
    assert np.linalg.norm(got - ref) <= 40 * (N + 1) * U24 / eps * np.linalg.norm(ref)
    assert abs(st.tdvp.e_mean_re - info["E"].real) <= 1e-5 * abs(info["E"])
    assert abs(complex(st.lambda_re, st.lambda_im) - lam) <= 1e-12
    w = np.abs(1 - info["rho"]) ** 2
    assert abs(st.ess - w.sum() ** 2 / (w * w).sum()) <= 1e-6 * n


def test_excited_search_exact_sums_reaches_e1():
    """Exact sums on the GPU (all states, Born weights of psi and phi): from the oracle's
    ground state of the N = 8 chain (J = h = 1), 120 steps of the search (dt 0.05, shift
    1e-3) bring <Psi|H|Psi>/<Psi|Psi> (oracle enumeration of the GPU's parameters) within
    1e-3 of the first excited energy of dense ED."""
    N, M, J, h = 8, 8, 1.0, 1.0
    ev = _e_levels(N, J, h)
    phi = _ground_state(N, M, J, h, 120)
    psi0 = inputs.rbm_params(N, M, 0.1, seed=77)
    ctx = _ctx(N, J, h, 256)
    try:
        vmc.vmc_set_params(ctx, 0, psi0)
        vmc.vmc_set_params(ctx, 1, phi)
        opts = vmc.make_tdvp_opts(gamma=1.0, shift=1e-3, exact=1)
        for _ in range(120):
            st = vmc.vmc_excited_step(ctx, 0, 1, 0.05, opts)
        psi = vmc.vmc_get_params(ctx, 0)
        assert np.array_equal(vmc.vmc_get_params(ctx, 1), phi)
    finally:
        vmc.vmc_destroy(ctx)
    E, _ = excited.exact_excited_energy(T, N, 1, J, h, M, psi, phi)
    assert abs(E.real - ev[1]) <= 1e-3 * abs(ev[1]), (E.real, ev[:3])
    assert abs(st.tdvp.e_mean_re - E.real) <= 1e-4 * abs(E.real)


def test_excited_search_monte_carlo_reaches_e1():
    """Monte Carlo: lambda from 256 x 200 Metropolis samples of |phi|^2 and the SR step of
    Psi from 256 x 200 importance-weighted samples of |psi|^2 every step (the 1D workload's
    sizes, N = 10): within 300 steps the exact energy of Psi is within 2e-3 of E_1.
    Psi does not change when a multiple of phi is added to psi, so nothing holds psi's
    component along phi in place: under Monte Carlo noise it grows, and with it the spread
    of the importance weights (the effective sample size falls to a few per cent of the
    samples here); the estimate stays unbiased, only noisier."""
    N, M, J, h = 10, 10, 1.0, 1.0
    ev = _e_levels(N, J, h)
    phi = _ground_state(N, M, J, h, 150)
    psi0 = inputs.rbm_params(N, M, 0.1, seed=77)
    ctx = _ctx(N, J, h, 256, spc=200)
    try:
        vmc.vmc_set_params(ctx, 0, psi0)
        vmc.vmc_set_params(ctx, 1, phi)
        vmc.vmc_set_chains(ctx, 0, inputs.random_spins(256, N, seed=8))
        vmc.vmc_set_chains(ctx, 1, inputs.random_spins(256, N, seed=9))
        opts = vmc.make_tdvp_opts(gamma=1.0, shift=1e-3)
        for _ in range(300):
            st = vmc.vmc_excited_step(ctx, 0, 1, 0.05, opts)
        psi = vmc.vmc_get_params(ctx, 0)
    finally:
        vmc.vmc_destroy(ctx)
    E, _ = excited.exact_excited_energy(T, N, 1, J, h, M, psi, phi)
    assert abs(E.real - ev[1]) <= 2e-3 * abs(ev[1]), (E.real, ev[:3])
    assert 0.005 * 256 * 200 < st.ess <= 256 * 200
