"""GPU parity of the regularised TDVP right-hand side and the adaptive Heun integrator
(vmc_tdvp_rhs, vmc_tdvp_step) with the FP64 oracle (oracle/tdvp.py), through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import tdvp
from paper_2108_03409_b300 import inputs, vmc

from gpu_helpers import context, cplx, lattice, to_dev_spins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T = inputs.MODEL_TFIM
U24 = 2.0 ** -24


def _gpu_rhs(ctx, s, opts, P, weights=None):
    out = torch.zeros((P, 2), dtype=torch.float64, device="cuda")
    w = None if weights is None else torch.from_numpy(np.ascontiguousarray(weights)).cuda()
    st = vmc.vmc_tdvp_rhs(ctx, 0, opts, out, spins=None if s is None else to_dev_spins(s),
                          weights=w)
    return cplx(out), st


@pytest.mark.parametrize("gamma,eps_pinv,soft,eps_snr",
                         [(1j, 1e-6, 1, 2.0), (1j, 1e-3, 0, 0.0), (1.0, 1e-8, 1, 0.0)],
                         ids=["real_soft_snr", "real_hard", "imag_soft"])
def test_tdvp_core_matches_oracle_on_the_same_fp32_inputs(gamma, eps_pinv, soft, eps_snr):
    """The FP64 core (weighted moments, S and Q Grams, Jacobi eigen-decomposition, SNR,
    damped inverse) against the oracle fed the GPU's own FP32 log-derivatives and local
    energies: the two differ by FP64 rounding only, amplified at most by the largest
    damped inverse eigenvalue: |d thetadot| <= 1e-12 * lambda_1 * max lambda^+ * |thetadot|
    (plus the same for F).  Samples: 4096 Metropolis-like random configurations of the
    N = 8 chain (P = 80), uniform weights (Monte Carlo)."""
    N, M, n = 8, 8, 4096
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.2, seed=71)
    s = inputs.random_spins(n, N, seed=72)
    with context(lattice(T, N, 1, 1.0, 0.9, 1), n_chains=n, solver=vmc.SOLVER_CG, tdvp=1) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        sd = to_dev_spins(s)
        e = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_local_energy(ctx, 0, sd, e)
        O = torch.zeros((n, P, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_grad(ctx, 0, sd, e, O, None)
        opts = vmc.make_tdvp_opts(gamma=gamma, eps_pinv=eps_pinv, pinv_soft=soft, eps_snr=eps_snr)
        got, st = _gpu_rhs(ctx, s, opts, P)
        Og, Eg = cplx(O), cplx(e)
    ref, info = tdvp.tdvp_rhs(Og, Eg, gamma=gamma, eps_pinv=eps_pinv, soft=bool(soft),
                              eps_snr=eps_snr)
    lam = info["lam"]
    amp = np.max(np.abs(lam)) * np.max(np.abs(info["lam_plus"]))
    assert st.jacobi_off <= 1e-13 and st.jacobi_sweeps < 40
    assert abs(st.lam_max - np.max(np.abs(lam))) <= 1e-12 * np.max(np.abs(lam))
    assert abs(st.lam_min - np.min(lam)) <= 1e-12 * np.max(np.abs(lam))
    err = np.linalg.norm(got - ref)
    assert err <= 1e-12 * amp * np.linalg.norm(ref) + 1e-14, (err, amp, np.linalg.norm(ref))
    assert abs(st.e_mean_re - np.mean(Eg).real) <= 1e-12 * abs(np.mean(Eg))


def test_tdvp_rhs_end_to_end_against_fp64_oracle():
    """The whole right-hand side from the spins (FP32 tanh theta and E_loc inside) against
    the oracle's FP64 O_k and E_loc.  The FP32 inputs carry relative errors of about
    (N + 1) 2^-24 (theta) and 2^-20 (E_loc); the soft cutoff bounds the amplification by
    the damped inverse at about 1 / eps_pinv, so
        |d thetadot| / |thetadot| <= 40 (N + 1) 2^-24 / eps_pinv."""
    N, M, n, eps = 8, 8, 4096, 1e-3
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.2, seed=73)
    s = inputs.random_spins(n, N, seed=74)
    with context(lattice(T, N, 1, 1.0, 0.9, 1), n_chains=n, solver=vmc.SOLVER_CG, tdvp=1) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        got, st = _gpu_rhs(ctx, s, vmc.make_tdvp_opts(gamma=1j, eps_pinv=eps), P)
    O = oracle.ok(N, M, p, s)
    E = oracle.eloc(T, N, 1, 1.0, 0.9, M, p, s)
    ref, _ = tdvp.tdvp_rhs(O, E, gamma=1j, eps_pinv=eps)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 40 * (N + 1) * U24 / eps, rel


def test_exact_sums_product_state_precession():
    """Exact enumeration on the GPU (all 2^N states, Born weights): the product state under
    H = -h sum X precesses as da/dt = -i h sinh(2a), and b, W get no velocity (their O_k
    vanish); FP32 inputs bound the agreement at 1e-5 relative."""
    N, h = 8, 0.7
    M = N
    P = N + M + N * M
    p = np.zeros(P, np.complex128)
    rng = np.random.default_rng(4)
    p[:N] = rng.normal(0, 0.4, N) + 1j * rng.normal(0, 0.4, N)
    with context(lattice(T, N, 1, 0.0, h, 1), n_chains=256, solver=vmc.SOLVER_CG, tdvp=1) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        got, st = _gpu_rhs(ctx, None, vmc.make_tdvp_opts(gamma=1j, eps_pinv=1e-6, pinv_soft=0,
                                                         exact=1), P)
    ref = -1j * h * np.sinh(2 * p[:N])
    assert np.max(np.abs(got[:N] - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert np.max(np.abs(got[N:])) <= 1e-6 * np.max(np.abs(ref))
    assert st.e_stderr == 0.0


def test_exact_sums_match_oracle_and_weights_path():
    """Exact sums of a generic RBM (N = 8, J = 1, h = 0.8): the context's own enumeration
    equals vmc_tdvp_rhs given all states and the oracle's Born weights, and both agree with
    the oracle's exact right-hand side to the FP32 input bound of the test above."""
    N, M, eps = 8, 8, 1e-3
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.3, seed=75)
    s_all = oracle.all_states(N)
    w = oracle.born_weights(oracle.logpsi(N, M, p, s_all))
    opts = vmc.make_tdvp_opts(gamma=1j, eps_pinv=eps, exact=1)
    with context(lattice(T, N, 1, 1.0, 0.8, 1), n_chains=256, solver=vmc.SOLVER_CG, tdvp=1) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        a, sa = _gpu_rhs(ctx, None, opts, P)
        b, sb = _gpu_rhs(ctx, s_all, opts, P, weights=w)
    ref, info = tdvp.exact_tdvp_rhs(T, N, 1, 1.0, 0.8, M, p, gamma=1j, eps_pinv=eps)
    bound = 40 * (N + 1) * U24 / eps
    assert np.linalg.norm(a - b) <= bound * np.linalg.norm(ref)
    assert np.linalg.norm(a - ref) <= bound * np.linalg.norm(ref)
    assert abs(sa.e_mean_re - info["E"].real) <= 1e-5 * abs(info["E"])


def test_sr_limit_equals_the_shifted_solve():
    """gamma = 1, no cutoff, shift nu: thetadot = -(S + nu diag S)^-1 F, the SR update the
    dense solvers compute; checked against the oracle's Cholesky solve on the same samples
    (FP32 inputs; N = 6, alpha = 1: P = 48 against 64 basis states)."""
    N, M, n, nu = 6, 6, 4096, 1e-1
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.3, seed=76)
    s = inputs.random_spins(n, N, seed=77)
    with context(lattice(T, N, 1, 1.0, 1.0, 1), n_chains=n, solver=vmc.SOLVER_CG, tdvp=1) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        got, _ = _gpu_rhs(ctx, s, vmc.make_tdvp_opts(gamma=1.0, shift=nu), P)
    O = oracle.ok(N, M, p, s)
    E = oracle.eloc(T, N, 1, 1.0, 1.0, M, p, s)
    S, F, _ = oracle.sr_matrices(O, E)
    ref = -oracle.cholesky_solve(oracle.shift(S, nu, 0), F)
    cond = np.linalg.cond(oracle.shift(S, nu, 0))
    assert np.linalg.norm(got - ref) <= 40 * (N + 1) * U24 * cond * np.linalg.norm(ref)


def test_adaptive_heun_step_exact_matches_oracle_and_conserves_energy():
    """vmc_tdvp_step with exact sums against the oracle's adaptive Heun step from the same
    parameters (first step: same accepted size to 1e-5, same parameters to the FP32 input
    bound), then 15 real-time steps whose exact energy stays within 1e-4 of the start (the
    oracle's own integrator drifts by 2e-5 over these steps at this tolerance, and by
    8.6e-4 at eps_step = 1e-5: the drift is the integration error).  The accepted size is
    tau (eps/delta)^(1/3) after the retries, and delta, the Fisher-norm distance of one full
    and two half Heun steps, is a difference of two integrations of a right-hand side
    formed from FP32 log-derivatives and local energies: two FP32 evaluations of the same
    local energies that both agree with FP64 to 2e-7 (a log-sum and a product of the
    factors) move the accepted size by 1.8e-6 on this case.  A wrong order or norm in the
    step-size rule changes it by far more than 1e-5."""
    N, M, J, h, eps, step_eps = 6, 6, 1.0, 0.8, 1e-4, 1e-7
    P = N + M + N * M
    p = inputs.rbm_params(N, M, 0.3, seed=11)
    opts = vmc.make_tdvp_opts(gamma=1j, eps_pinv=eps, exact=1, eps_step=step_eps)
    E = lambda q: oracle.exact_energy(T, N, 1, J, h, M, q)[0].real
    with context(lattice(T, N, 1, J, h, 1), n_chains=128, solver=vmc.SOLVER_CG, tdvp=1) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        t1, tau1, st1 = vmc.vmc_tdvp_step(ctx, 0, opts, 0.0, 0.01)
        y1 = vmc.vmc_get_params(ctx, 0)
        t, tau = t1, tau1
        for _ in range(15):
            t, tau, st = vmc.vmc_tdvp_step(ctx, 0, opts, t, tau)
        y = vmc.vmc_get_params(ctx, 0)
    f = lambda y_, t_: tdvp.exact_tdvp_rhs(T, N, 1, J, h, M, y_, gamma=1j, eps_pinv=eps)
    norm = lambda v, info: tdvp.fisher_norm(v, info["S"])
    yo, to, tauo, used, delta, retries = tdvp.adaptive_heun_step(f, p, 0.0, 0.01, step_eps, norm)
    assert st1.rhs_evals == 1 + 4 * (st1.retries + 1) and retries == st1.retries
    assert abs(st1.tau_used - used) <= 1e-5 * used and abs(t1 - to) <= 1e-5 * to
    assert np.linalg.norm(y1 - yo) <= 40 * (N + 1) * U24 / eps * np.linalg.norm(yo - p)
    e0 = E(p)
    assert abs(E(y) - e0) <= 1e-4 * abs(e0), (E(y), e0)
    assert t > 0.03


def test_adaptive_heun_step_monte_carlo_real_time():
    """Monte Carlo right-hand sides (each of the five evaluations samples the chains anew,
    SNR damping on): a few real-time steps of the N = 10 chain at h = 1 after a quench from
    the near-uniform state keep the exact energy of the parameters within 3 % of its start
    (the MC noise of 51 200 samples per evaluation, not an integration error) and report
    a finite SNR."""
    N, M, J, h = 10, 10, 1.0, 1.0
    p = inputs.rbm_params(N, M, 0.1, seed=1234)
    opts = vmc.make_tdvp_opts(gamma=1j, eps_pinv=1e-4, eps_snr=2.0, eps_step=1e-4, tau_max=0.02)
    E = lambda q: oracle.exact_energy(T, N, 1, J, h, M, q)[0].real
    with context(lattice(T, N, 1, J, h, 1), n_chains=256, samples_per_chain=200, therm_sweeps=20,
                 solver=vmc.SOLVER_CG, tdvp=1) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, inputs.random_spins(256, N, seed=5))
        t, tau = 0.0, 0.005
        for _ in range(4):
            t, tau, st = vmc.vmc_tdvp_step(ctx, 0, opts, t, tau)
            assert st.snr_min > 0 and np.isfinite(st.snr_min)
        y = vmc.vmc_get_params(ctx, 0)
    e0 = E(p)
    assert abs(E(y) - e0) <= 0.03 * abs(e0)
    assert t > 0 and np.linalg.norm(y - p) > 0


def test_tdvp_needs_its_workspaces():
    with context(lattice(T, 8, 1, 1.0, 1.0, 1), n_chains=64, solver=vmc.SOLVER_CG) as ctx:
        out = torch.zeros((80, 2), dtype=torch.float64, device="cuda")
        with pytest.raises(vmc.VmcError) as ei:
            vmc.vmc_tdvp_rhs(ctx, 0, vmc.make_tdvp_opts(exact=1), out)
        assert ei.value.status == vmc.VMC_ERR_STATE
    with context(lattice(T, 10, 1, 1.0, 1.0, 1), n_chains=64, solver=vmc.SOLVER_CG, tdvp=1) as ctx:
        out = torch.zeros((120, 2), dtype=torch.float64, device="cuda")
        with pytest.raises(vmc.VmcError) as ei:                 # 2^10 > 64 samples
            vmc.vmc_tdvp_rhs(ctx, 0, vmc.make_tdvp_opts(exact=1), out)
        assert ei.value.status == vmc.VMC_ERR_ARG
