"""Pins of the CNN-ELU ansatz oracle (oracle/cnn.py, Eq. gs_nqs): symmetry, finite
differences, a dense Hamiltonian built independently, the Metropolis chain's stationary
distribution, and the paper's ground-state recipe reaching the Jordan-Wigner energy."""
import numpy as np
from scipy.stats import chi2

import oracle
from oracle import cnn
from paper_2108_03409_b300 import inputs

from test_oracle_pins import _dense_h, _state_index, jordan_wigner_e0

T = inputs.MODEL_TFIM


def _params(N, alpha, seed, sigma=0.3):
    return np.random.default_rng(seed).normal(0.0, sigma, cnn.nparams(N, alpha))


def test_translation_invariance():
    """Summing over all translations makes log psi invariant under every shift of s."""
    N, alpha = 9, 3
    p = _params(N, alpha, 1)
    s = inputs.random_spins(50, N, seed=2)
    lp = cnn.logpsi(N, alpha, p, s)
    for k in range(1, N):
        assert np.max(np.abs(cnn.logpsi(N, alpha, p, np.roll(s, k, axis=1)) - lp)) <= 1e-12


def test_log_derivatives_by_finite_differences():
    N, alpha = 7, 2
    p = _params(N, alpha, 3)
    s = inputs.random_spins(40, N, seed=4)
    O = cnn.ok(N, alpha, p, s)
    eps = 1e-6
    for k in range(p.size):
        dp = np.zeros_like(p)
        dp[k] = eps
        fd = (cnn.logpsi(N, alpha, p + dp, s) - cnn.logpsi(N, alpha, p - dp, s)) / (2 * eps)
        assert np.max(np.abs(fd - O[:, k])) <= 1e-7 * max(1.0, np.max(np.abs(O[:, k])))


def test_local_energy_is_h_psi_over_psi():
    N, alpha, J, h = 8, 2, 1.0, 0.7
    p = _params(N, alpha, 5)
    s = oracle.all_states(N)
    psi = np.exp(cnn.logpsi(N, alpha, p, s))
    ref = (_dense_h(T, N, 1, J, h) @ psi) / psi
    got = cnn.eloc(T, N, 1, J, h, alpha, p, s)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_metropolis_is_stationary_on_psi2():
    """2048 chains x 25 single-flip sweeps of the N = 6 chain: the final states' histogram
    against the exact |psi|^2 (chi-square, p-value > 1e-3)."""
    N, alpha, C = 6, 2, 2048
    p = _params(N, alpha, 6, sigma=0.5)
    s0 = inputs.random_spins(C, N, seed=7)
    fin, _, _ = cnn.metropolis(N, alpha, p, s0, seed=8, n_sweeps=25)
    states = oracle.all_states(N)
    prob = np.exp(2 * cnn.logpsi(N, alpha, p, states))
    prob /= prob.sum()
    counts = np.bincount(_state_index(fin), minlength=len(states))
    exp = C * prob
    keep = exp >= 5
    stat = np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep])
    rest_o, rest_e = counts[~keep].sum(), exp[~keep].sum()
    dof = keep.sum() - 1
    if rest_e > 0:
        stat += (rest_o - rest_e) ** 2 / rest_e
        dof += 1
    assert chi2.sf(stat, dof) > 1e-3, (stat, dof)


def test_ground_state_recipe_reaches_jordan_wigner():
    """The paper's recipe (SR, tau = 1e-2, diagonal shift nu = 10 * 0.95^n, pseudo-inverse
    cutoff 1e-8) with exact sums on the L = 10 chain at g = 0.7, alpha = 2: within 250
    steps the energy is within 1e-3 of the Jordan-Wigner value."""
    N, alpha, J, g = 10, 2, 1.0, 0.7
    E0 = jordan_wigner_e0(N, J, g)
    p = np.random.default_rng(1).normal(0, 0.1, cnn.nparams(N, alpha))
    s = oracle.all_states(N)
    for it in range(250):
        lp = cnn.logpsi(N, alpha, p, s)
        w = np.exp(2 * (lp - lp.max()))
        w /= w.sum()
        E = cnn.eloc(T, N, 1, J, g, alpha, p, s)
        O = cnn.ok(N, alpha, p, s)
        Em = np.sum(w * E)
        Ob = O - (w @ O)[None, :]
        S = (Ob.T * w) @ Ob
        F = Ob.T @ (w * (E - Em))
        St = S + 10 * 0.95 ** it * np.diag(np.diag(S))
        lam, V = np.linalg.eigh(St)
        lplus = np.where(np.abs(lam) / np.abs(lam).max() >= 1e-8, 1 / lam, 0.0)
        p = p - 0.01 * (V @ (lplus * (V.T @ F)))
        if abs(Em - E0) / abs(E0) <= 1e-3:
            break
    assert abs(Em - E0) / abs(E0) <= 1e-3, (it, Em, E0)
