"""Pins of the TDVP oracle (oracle/tdvp.py): the regularised right-hand side and the
adaptive Heun integrator, checked against closed forms and invariants of the paper's
equations rather than against themselves (sections "Unitary dynamics", "Regularization
to invert the (quantum) Fisher matrix", "Utilities")."""
import numpy as np
import pytest

import oracle
from oracle import tdvp
from paper_2108_03409_b300 import inputs

T = inputs.MODEL_TFIM


def _product_state(N, seed):
    """RBM with W = 0 and b = 0: psi(s) = prod_i exp(a_i s_i), a product state."""
    M = N
    p = np.zeros(N + M + N * M, np.complex128)
    rng = np.random.default_rng(seed)
    p[:N] = rng.normal(0, 0.4, N) + 1j * rng.normal(0, 0.4, N)
    return p, M


@pytest.mark.parametrize("gamma", [1j, 1.0], ids=["real_time", "imaginary_time"])
def test_product_state_precession_closed_form(gamma):
    """Under H = -h sum X_i (J = 0) a product state stays a product state; each spin's
    amplitude ratio r = c_up / c_dn = exp(2 a) obeys dr/dt = -gamma * (-h) (1 - r^2)
    (from i dc/dt = H c for gamma = i, dc/dtau = -H c for gamma = 1), i.e.
        da/dt = -gamma h sinh(2 a).
    The manifold contains the exact flow, so the TDVP must reproduce it; the b and W
    directions have O = 0 (zero rows of S) and must get zero velocity."""
    N, h = 5, 0.7
    p, M = _product_state(N, 3)
    td, info = tdvp.exact_tdvp_rhs(T, N, 1, 0.0, h, M, p, gamma=gamma, eps_pinv=1e-10, soft=False)
    ref = -gamma * h * np.sinh(2 * p[:N])
    assert np.max(np.abs(td[:N] - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(td[N:])) <= 1e-12


def _rbm(N, M, sigma, seed):
    return inputs.rbm_params(N, M, sigma, seed=seed)


def test_energy_conservation_and_descent():
    """dE/dt = 2 Re(F^H thetadot) (holomorphic ansatz: dE/dtheta_k = conj(F_k)).  With
    thetadot = -gamma S^+ F and S^+ Hermitian PSD (any real damping of the eigenvalues),
    the real-time flow (gamma = i) conserves E and the imaginary-time flow (gamma = 1)
    lowers it at the rate -2 sum_k lambda^+_k |rho_k|^2.  Checked against central finite
    differences of the exact energy along thetadot."""
    N, M, J, h = 6, 6, 1.0, 0.8
    p = _rbm(N, M, 0.3, 11)
    E = lambda q: oracle.exact_energy(T, N, 1, J, h, M, q)[0].real
    eps = 1e-5
    for gamma in (1j, 1.0):
        for kw in (dict(eps_pinv=1e-6, soft=True), dict(eps_pinv=1e-3, soft=False)):
            td, info = tdvp.exact_tdvp_rhs(T, N, 1, J, h, M, p, gamma=gamma, **kw)
            dEdt = (E(p + eps * td) - E(p - eps * td)) / (2 * eps)
            rate = -2 * np.real(gamma) * np.sum(info["lam_plus"] * np.abs(info["rho"]) ** 2)
            scale = np.sum(np.abs(info["lam_plus"]) * np.abs(info["rho"]) ** 2)
            assert abs(dEdt - rate) <= 1e-6 * scale + 1e-10, (gamma, kw, dEdt, rate)
            if gamma == 1.0:
                assert rate < 0


def test_pseudo_inverse_is_the_inverse_without_cutoff():
    """eps_pinv = 0 on a well-conditioned S: thetadot = -gamma S^-1 F (numpy solve).
    (P = 20 parameters against 64 basis states, so S has full rank.)"""
    N, M = 6, 2
    p = _rbm(N, M, 0.3, 5)
    s = inputs.random_spins(3000, N, seed=6)
    O = oracle.ok(N, M, p, s)
    E = oracle.eloc(T, N, 1, 1.0, 1.0, M, p, s)
    for gamma in (1j, 1.0):
        td, info = tdvp.tdvp_rhs(O, E, gamma=gamma)
        ref = -gamma * np.linalg.solve(info["S"], info["F"])
        assert np.linalg.cond(info["S"]) < 1e8
        assert np.linalg.norm(td - ref) <= 1e-9 * np.linalg.norm(ref)


def test_hard_cutoff_drops_exactly_the_small_eigenvalues():
    """Eq. pinv_cutoff: in the eigenbasis, components with |lambda/lambda_1| < eps get no
    velocity and the others -gamma rho_k / lambda_k."""
    N, M = 4, 4
    p = _rbm(N, M, 0.3, 7)
    s = inputs.random_spins(400, N, seed=8)
    O = oracle.ok(N, M, p, s)
    E = oracle.eloc(T, N, 1, 1.0, 1.0, M, p, s)
    td, info = tdvp.tdvp_rhs(O, E, gamma=1j, eps_pinv=1e-2, soft=False)
    lam, V, rho = info["lam"], info["V"], info["rho"]
    c = V.conj().T @ td
    small = np.abs(lam) / np.max(np.abs(lam)) < 1e-2
    assert small.any() and (~small).any()
    assert np.max(np.abs(c[small])) <= 1e-12 * np.max(np.abs(c))
    assert np.allclose(c[~small], -1j * rho[~small] / lam[~small], rtol=1e-10, atol=0)


def test_snr_variance_identity_and_noise_meaning():
    """The per-sample variance of rho_k(s) equals (V^H Q V)_kk - |rho_k|^2 with the energy-
    weighted Gram Q = <|E - <E>|^2 conj(Obar) Obar^T> (the way the CUDA path forms it); and
    SNR = |rho_k| / sqrt(var / n) is the signal-to-noise ratio of the Monte Carlo estimate:
    over 300 independent sets of n = 400 exact draws from |psi|^2, the spread of the
    estimates of rho_k (projected on the exact eigenbasis) matches sqrt(var / n) within 15 %
    for the components whose noise is at least 5 % of the largest."""
    N, M, J, h = 5, 5, 1.0, 0.9
    p = _rbm(N, M, 0.3, 13)
    s_all = oracle.all_states(N)
    w = oracle.born_weights(oracle.logpsi(N, M, p, s_all))
    E_all = oracle.eloc(T, N, 1, J, h, M, p, s_all)
    O_all = oracle.ok(N, M, p, s_all)
    td, info = tdvp.tdvp_rhs(O_all, E_all, w, gamma=1j, eps_snr=1.0, n_eff=1)
    S, F, Em, Ob, f, ww = tdvp.tdvp_matrices(O_all, E_all, w)
    V = info["V"]
    Q = (Ob.conj().T * (ww * np.abs(E_all - Em) ** 2)[None, :]) @ Ob
    var_gram = np.real(np.einsum("lk,lm,mk->k", V.conj(), Q, V)) - np.abs(info["rho"]) ** 2
    assert np.allclose(info["rho_var"], var_gram, rtol=1e-9, atol=1e-12 * np.max(var_gram))
    rng = np.random.default_rng(3)
    n, R = 400, 300
    est = []
    for _ in range(R):
        idx = rng.choice(len(s_all), size=n, p=w)
        _, Fm, _, _, _, _ = tdvp.tdvp_matrices(O_all[idx], E_all[idx])
        est.append(V.conj().T @ Fm)
    est = np.array(est)
    spread = np.sqrt(np.mean(np.abs(est - est.mean(axis=0)) ** 2, axis=0))
    pred = np.sqrt(info["rho_var"] / n)
    # (components whose noise is below 5 % of the largest are dominated by the second-order
    # terms of the sample-mean centring, which the first-order variance does not describe)
    big = pred > 0.05 * pred.max()
    assert big.sum() >= 10
    assert np.all(np.abs(spread[big] / pred[big] - 1) <= 0.15), (spread / pred)[big]


def test_snr_damping_scales_with_sqrt_n():
    """Duplicating every sample leaves rho and the variance unchanged and doubles n, so the
    SNR grows by sqrt(2) and the damping 1/(1 + (eps/SNR)^6) follows; scaling E by a
    constant scales rho and its noise alike (the damping is unchanged).  (Full-rank S:
    P = 20 against 64 basis states, so the eigenbasis is unique up to phases.)"""
    N, M = 6, 2
    p = _rbm(N, M, 0.3, 21)
    s = inputs.random_spins(300, N, seed=22)
    O = oracle.ok(N, M, p, s)
    E = oracle.eloc(T, N, 1, 1.0, 1.0, M, p, s)
    eps = 3.0
    _, a = tdvp.tdvp_rhs(O, E, gamma=1j, eps_snr=eps)
    _, b = tdvp.tdvp_rhs(np.concatenate([O, O]), np.concatenate([E, E]), gamma=1j, eps_snr=eps)
    _, c = tdvp.tdvp_rhs(O, 7.0 * E, gamma=1j, eps_snr=eps)
    snr_a = np.abs(a["rho"]) / np.sqrt(a["rho_var"] / 300)
    da = a["lam_plus"] * a["lam"]
    db = b["lam_plus"] * b["lam"]
    assert np.allclose(da, 1 / (1 + (eps / snr_a) ** 6), rtol=1e-9)
    assert np.allclose(db, 1 / (1 + (eps / (np.sqrt(2) * snr_a)) ** 6), rtol=1e-7)
    assert np.allclose(c["lam_plus"], a["lam_plus"], rtol=1e-9)


def test_adaptive_heun_order_and_accuracy():
    """y' = -i omega y: the two-half-step Heun solution differs from the one-step solution
    by O(tau^3), so the accepted steps scale like eps^(1/3) and the end point at t = 2 is
    accurate to a small multiple of the accumulated tolerance."""
    om = np.array([1.0, 2.5, -0.7])
    f = lambda y, t: (-1j * om * y, None)
    norm = lambda v, info: float(np.linalg.norm(v))
    res = {}
    for eps in (1e-6, 1e-9):
        y, t, tau, steps = np.ones(3, np.complex128), 0.0, 0.01, 0
        while t < 2.0 - 1e-12:
            tau = min(tau, 2.0 - t)
            y, t, tau, used, delta, _ = tdvp.adaptive_heun_step(f, y, t, tau, eps, norm)
            assert delta <= eps
            steps += 1
        res[eps] = steps
        err = np.linalg.norm(y - np.exp(-1j * om * 2.0))
        assert err <= 10 * steps * eps, (eps, err, steps)
    ratio = res[1e-9] / res[1e-6]
    assert 7.0 <= ratio <= 13.0, ratio          # (1e3)^(1/3) = 10


def test_adaptive_heun_product_state_trajectory_and_energy():
    """Integrated with the exact right-hand side and the Fisher norm, the product state
    follows the closed-form precession c(t) = exp(i h t X) c(0) per spin (real time,
    J = 0), and a generic RBM conserves its energy along the real-time flow to the
    integrator's tolerance."""
    N, h = 4, 0.7
    p, M = _product_state(N, 9)
    a0 = p[:N].copy()
    f = lambda y, t: tdvp.exact_tdvp_rhs(T, N, 1, 0.0, h, M, y, gamma=1j, eps_pinv=1e-10,
                                         soft=False)
    norm = lambda v, info: tdvp.fisher_norm(v, info["S"])
    y, t, tau = p.copy(), 0.0, 0.01
    while t < 0.6 - 1e-12:
        tau = min(tau, 0.6 - t)
        y, t, tau, *_ = tdvp.adaptive_heun_step(f, y, t, tau, 1e-9, norm)
    c, s_ = np.cos(h * t), np.sin(h * t)
    r = (c * np.exp(a0) + 1j * s_ * np.exp(-a0)) / (1j * s_ * np.exp(a0) + c * np.exp(-a0))
    assert np.max(np.abs(np.exp(2 * y[:N]) - r)) <= 1e-5 * np.max(np.abs(r))
    # energy conservation of a generic RBM
    N, M, J, h = 6, 6, 1.0, 0.8
    p = _rbm(N, M, 0.3, 11)
    E = lambda q: oracle.exact_energy(T, N, 1, J, h, M, q)[0].real
    f = lambda y, t: tdvp.exact_tdvp_rhs(T, N, 1, J, h, M, y, gamma=1j, eps_pinv=1e-8)
    y, t, tau, e0 = p.copy(), 0.0, 0.005, E(p)
    while t < 0.3 - 1e-12:
        tau = min(tau, 0.3 - t)
        y, t, tau, *_ = tdvp.adaptive_heun_step(f, y, t, tau, 1e-6, norm)
    assert abs(E(y) - e0) <= 1e-4 * abs(e0), (E(y), e0)
    assert np.linalg.norm(y - p) > 1e-2          # the state did move
