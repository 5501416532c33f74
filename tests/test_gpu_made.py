"""GPU parity of the learned proposal (masked autoregressive MLP) with the FP64 oracle,
and stationarity of the independent Metropolis-Hastings chains it drives."""
import numpy as np
import pytest

import oracle
from paper_2108_03409_b300 import inputs
from paper_2108_03409_b300 import stats, vmc

from gpu_helpers import context, cplx, lattice, to_dev_spins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T = inputs.MODEL_TFIM

# FP32 forward: |d log q| <= LOGQ_ABS_PER_SITE * N + LOGQ_REL * |log q| (each of the N terms
# log sigma(s z) carries FP32 rounding of z, a sum over <= H + N products)
LOGQ_ABS_PER_SITE = 2e-6
LOGQ_REL = 1e-6


@pytest.mark.parametrize("N,H,scale", [(10, 32, 1.0), (36, 64, 1.5), (144, 256, 1.0)])
def test_made_logq_matches_oracle(N, H, scale):
    p = inputs.made_params(N, H, seed=3, scale=scale)
    s = inputs.random_spins(300, N, seed=4)
    with context(lattice(T, N, 1, 1.0, 1.0, 1), n_chains=300, solver=vmc.SOLVER_CG,
                 made_hidden=H) as ctx:
        vmc.vmc_made_set_params(ctx, 0, p)
        out = torch.zeros(300, dtype=torch.float32, device="cuda")
        vmc.vmc_made_logq(ctx, 0, to_dev_spins(s), out)
        got = out.cpu().numpy().astype(np.float64)
        back = vmc.vmc_made_get_params(ctx, 0, p.size)
    assert np.array_equal(back, p)
    ref = oracle.made_forward(N, H, p.astype(np.float64), s)
    assert np.all(np.abs(got - ref) <= LOGQ_ABS_PER_SITE * N + LOGQ_REL * np.abs(ref))


@pytest.mark.parametrize("N,H,n", [(10, 32, 512), (36, 64, 1000), (144, 256, 4096)],
                         ids=["N10H32", "N36H64", "N144H256_batch4096"])
def test_made_grad_matches_oracle(N, H, n):
    """Backpropagation through the masked layers; the batch sum is FP32 (n terms), so the
    gradient error is stated relative to the largest gradient entry: n * 2^-24 * 8."""
    p = inputs.made_params(N, H, seed=5, scale=1.2)
    s = inputs.random_spins(n, N, seed=6)
    with context(lattice(T, N, 1, 1.0, 1.0, 1), n_chains=n, solver=vmc.SOLVER_CG,
                 made_hidden=H, made_batch=n) as ctx:
        vmc.vmc_made_set_params(ctx, 0, p)
        g = torch.zeros(p.size, dtype=torch.float32, device="cuda")
        loss = vmc.vmc_made_grad(ctx, 0, to_dev_spins(s), g)
        g = g.cpu().numpy().astype(np.float64)
    gref, Lref = oracle.made_grad(N, H, p.astype(np.float64), s)
    assert abs(loss - Lref) <= 1e-5 * abs(Lref)
    assert np.max(np.abs(g - gref)) <= n * 2.0 ** -24 * 8 * np.max(np.abs(gref)) + 1e-7
    assert np.all(g[gref == 0.0] == 0.0)          # masked entries stay exactly zero


def test_made_sampler_matches_oracle():
    """Same Philox stream: every draw equals the oracle's except where the oracle met a
    uniform within 1e-5 of sigma(z) (FP32 and FP64 may decide those differently)."""
    N, H, n = 36, 64, 512
    p = inputs.made_params(N, H, seed=7, scale=1.5)
    with context(lattice(T, 6, 6, 1.0, 1.0, 1), n_chains=n, solver=vmc.SOLVER_CG, made_hidden=H,
                 seed=11) as ctx:
        vmc.vmc_made_set_params(ctx, 0, p)
        s = torch.zeros((n, N), dtype=torch.int8, device="cuda")
        lq = torch.zeros(n, dtype=torch.float32, device="cuda")
        vmc.vmc_made_sample(ctx, 0, n, 5, s, lq)
        s = s.cpu().numpy()
        lq = lq.cpu().numpy().astype(np.float64)
    sref, lqref, margin = oracle.made_sample(N, H, p.astype(np.float64), n, seed=11, stream=0,
                                             round_=5)
    same = np.all(s == sref, axis=1)
    assert np.all(margin[~same] < 1e-5) and same.mean() >= 0.99
    assert np.all(np.abs(lq[same] - lqref[same]) <= LOGQ_ABS_PER_SITE * N + LOGQ_REL * np.abs(lqref[same]))


def test_adam_training_matches_oracle_steps():
    """Three Adam steps on the same batches: parameters agree with the FP64 oracle to the
    FP32 accuracy of the gradients (Adam normalises each step to ~lr)."""
    N, H, n, lr = 10, 32, 256, 1e-2
    p = inputs.made_params(N, H, seed=8)
    s = inputs.random_spins(3 * n, N, seed=9)
    with context(lattice(T, N, 1, 1.0, 1.0, 1), n_chains=n, solver=vmc.SOLVER_CG, made_hidden=H,
                 made_batch=n) as ctx:
        vmc.vmc_made_set_params(ctx, 0, p)
        vmc.vmc_proposal_train(ctx, 0, to_dev_spins(s), epochs=1, lr=lr)
        got = vmc.vmc_made_get_params(ctx, 0, p.size).astype(np.float64)
    th = p.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for t in range(3):
        g, _ = oracle.made_grad(N, H, th, s[t * n:(t + 1) * n])
        th, m, v = oracle.adam_step(th, m, v, g, t + 1, lr=lr)
    # entries whose gradient is tiny can take a full-size Adam step of either sign; compare
    # the well-determined ones tightly and all of them within the three-step bound
    assert np.max(np.abs(got - th)) <= 3 * 2 * lr
    g0, _ = oracle.made_grad(N, H, p.astype(np.float64), s[:n])
    big = np.abs(g0) > 1e-3 * np.max(np.abs(g0))
    assert np.median(np.abs(got - th)[big]) <= 1e-3 * lr


def test_learned_proposal_is_stationary_on_psi2():
    """Train q on samples of |psi|^2 (N = 10 TFIM chain), then run independent MH: the
    chains' final states are draws from |psi|^2 (chi-square at N = 10), and the acceptance
    is high because q approximates |psi|^2."""
    from scipy.stats import chi2
    N, M, H, C = 10, 10, 32, 16384
    p = inputs.rbm_params(N, M, 0.2, seed=101)
    q_init = inputs.made_params(N, H, seed=12)
    s0 = inputs.random_spins(C, N, seed=13)
    with context(lattice(T, N, 1, 1.0, 1.0, 1), n_chains=C, solver=vmc.SOLVER_CG, made_hidden=H,
                 made_batch=4096, seed=21) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, s0)
        train = torch.zeros((4 * C, N), dtype=torch.int8, device="cuda")
        vmc.vmc_sample(ctx, 0, 30, 4, train)                     # local Metropolis samples
        vmc.vmc_made_set_params(ctx, 0, q_init)
        loss = vmc.vmc_proposal_train(ctx, 0, train, epochs=30, lr=3e-3)
        acc = vmc.vmc_sample_learned(ctx, 0, 10)
        final = vmc.vmc_get_chains(ctx, 0, C, N)
    full = oracle.all_states(N)
    prob = oracle.born_weights(oracle.logpsi(N, M, p, full))
    entropy = -np.sum(prob * np.log(prob))
    assert loss <= entropy + 0.05                 # q close to |psi|^2 in KL
    assert acc >= 0.8
    idx = (((1 - final.astype(np.int64)) // 2) << np.arange(N)).sum(axis=1)
    counts = np.bincount(idx, minlength=1 << N)
    exp = prob * C
    order = np.argsort(exp)
    c_m, e_m, ac, ae = [], [], 0.0, 0.0
    for k in order:
        ac += counts[k]; ae += exp[k]
        if ae >= 5:
            c_m.append(ac); e_m.append(ae); ac = ae = 0.0
    c_m[-1] += ac; e_m[-1] += ae
    c_m, e_m = np.array(c_m), np.array(e_m)
    assert chi2.sf(np.sum((c_m - e_m) ** 2 / e_m), len(c_m) - 1) > 1e-3


def _series_stats(e, tau):
    """Mean and standard error of a [T][C] series with integrated autocorrelation tau."""
    n_rec, n_ch = e.shape
    return e.mean(), np.sqrt(e.var() / (n_rec * n_ch) * 2.0 * tau)


def test_learned_proposal_gain_over_local_moves():
    """What the trained proposal gains: on a peaked |psi|^2 (N = 12 TFIM chain, sigma = 0.35)
    single-flip chains decorrelate slowly; independent MH with q trained on their samples
    has a smaller integrated autocorrelation time of E_loc, while both samplers' <E> agree
    with exact enumeration and with each other within error bars."""
    N, M, H, C, R = 12, 12, 64, 8192, 120
    p = inputs.rbm_params(N, M, 0.35, seed=301)
    e_exact = oracle.exact_energy(T, N, 1, 1.0, 1.0, M, p)[0].real
    with context(lattice(T, N, 1, 1.0, 1.0, 1), n_chains=C, solver=vmc.SOLVER_CG,
                 made_hidden=H, made_batch=4096, seed=31) as ctx:
        vmc.vmc_set_params(ctx, 0, p)
        vmc.vmc_set_chains(ctx, 0, inputs.random_spins(C, N, seed=32))
        train = torch.zeros((16 * C, N), dtype=torch.int8, device="cuda")
        vmc.vmc_sample(ctx, 0, 300, 16, train)
        vmc.vmc_made_set_params(ctx, 0, inputs.made_params(N, H, seed=33))
        vmc.vmc_proposal_train(ctx, 0, train, epochs=20, lr=3e-3)
        el_loc = torch.zeros((R * C, 2), dtype=torch.float32, device="cuda")
        vmc.vmc_sample(ctx, 0, 0, R, None, None, el_loc)
        el_lrn = torch.zeros((R * C, 2), dtype=torch.float32, device="cuda")
        acc = vmc.vmc_sample_learned(ctx, 0, R, None, el_lrn)
    e_loc = cplx(el_loc).real.reshape(R, C)
    e_lrn = cplx(el_lrn).real.reshape(R, C)
    tau_loc = stats.integrated_autocorr_time(e_loc)
    tau_lrn = stats.integrated_autocorr_time(e_lrn)
    m_loc, err_loc = _series_stats(e_loc, tau_loc)
    m_lrn, err_lrn = _series_stats(e_lrn, tau_lrn)
    info = dict(tau_loc=tau_loc, tau_lrn=tau_lrn, acc=acc, m_loc=m_loc, m_lrn=m_lrn,
                err_loc=err_loc, err_lrn=err_lrn, exact=e_exact)
    assert acc >= 0.3, info
    assert tau_lrn < 0.7 * tau_loc, info
    assert abs(m_loc - e_exact) <= 4 * err_loc, info
    assert abs(m_lrn - e_exact) <= 4 * err_lrn, info
    assert abs(m_lrn - m_loc) <= 4 * np.hypot(err_loc, err_lrn), info
