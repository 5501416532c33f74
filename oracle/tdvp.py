"""FP64 oracle of the regularised TDVP right-hand side and the adaptive Heun integrator
(arXiv:2108.03409, sections "Unitary dynamics", "Regularization to invert the (quantum)
Fisher matrix" and "Utilities": TDVP and Stepper).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain numpy following the paper's
steps in its order; the eigendecomposition is numpy.linalg.eigh (a library primitive).

The equation solved is Eq. tdvp_util with the identity for [[.]] (holomorphic ansatz):
    S thetadot = -gamma F,   gamma = 1 (imaginary time, the SR step) or i (real time),
with S and F the connected correlators of Eq. qfm / Eq. force_vector under sample weights
w (1/n for Monte Carlo samples, the Born weights p(s) for exact enumeration).  S is
diagonalised, S = V diag(lambda) V^H, F is taken to its eigenbasis, rho = V^H F, and
    thetadot = -gamma V diag(lambda^+) rho,
with lambda^+ from the pseudo-inverse cutoff (Eq. pinv_cutoff, or its soft form) and the
signal-to-noise damping of the section "Eliminating noisy contributions".  Readings (the
paper leaves these open):
  * the two regularisations combine as a product of their damping factors:
        lambda^+ = 1/lambda * 1/(1 + (eps_pinv/|lambda/lambda_1|)^6) * 1/(1 + (eps_snr/SNR)^6)
    (soft), or the hard cutoff's 0/1 factor in place of the first one; lambda = 0 -> 0;
  * SNR(rho_k) = |rho_k| / sqrt(var_s(rho_k(s)) / n_eff), with the per-sample terms
    rho_k(s) = sum_l conj(V_lk) conj(Obar_l(s)) (E(s) - <E>), whose weighted mean is rho_k,
    and n_eff the number of Monte Carlo samples (no SNR damping with exact sums);
  * the optional diagonal shift is applied to S before the diagonalisation.

Parity status: tdvp_rhs, exact_tdvp_rhs and adaptive_heun_step are pinned in
tests/test_oracle_tdvp_pins.py (product-state precession closed form, energy conservation
of the real-time flow, the plain inverse for eps = 0, the hard cutoff, the SNR's sqrt(n)
scaling and scale invariance, the integrator's order and closed-form trajectories).
"""
from __future__ import annotations

import numpy as np

from . import all_states, born_weights, eloc, logpsi, ok


def tdvp_matrices(O: np.ndarray, E: np.ndarray, w=None):
    """Weighted S, F, <E>, the centred O and the per-sample force terms
    f_l(s) = conj(Obar_l(s)) (E(s) - <E>) (Eq. qfm, Eq. force_vector)."""
    O = np.asarray(O, dtype=np.complex128)
    E = np.asarray(E, dtype=np.complex128)
    n = O.shape[0]
    w = np.full(n, 1.0 / n) if w is None else np.asarray(w, np.float64) / np.sum(w)
    Em = np.sum(w * E)
    Ob = O - (w @ O)[None, :]
    S = (Ob.conj().T * w[None, :]) @ Ob
    f = Ob.conj() * (E - Em)[:, None]
    F = w @ f
    return S, F, Em, Ob, f, w


def damping(lam, rho=None, rho_var=None, n_eff=None, eps_pinv=0.0, soft=True, eps_snr=0.0):
    """lambda^+ of every eigenvalue (see the module docstring)."""
    lam = np.asarray(lam, np.float64)
    lam1 = np.max(np.abs(lam))
    r = np.abs(lam) / lam1 if lam1 > 0 else np.zeros_like(lam)
    with np.errstate(divide="ignore", invalid="ignore"):
        if eps_pinv > 0:
            if soft:
                d = np.where(r > 0, 1.0 / (1.0 + (eps_pinv / r) ** 6), 0.0)
            else:
                d = (r >= eps_pinv).astype(np.float64)
        else:
            d = (lam != 0).astype(np.float64)
        if eps_snr > 0:
            snr = np.abs(rho) / np.sqrt(rho_var / n_eff)
            d = d / (1.0 + (eps_snr / snr) ** 6)
        lp = np.where(lam != 0, d / lam, 0.0)
    return np.nan_to_num(lp, nan=0.0, posinf=0.0, neginf=0.0)


def tdvp_rhs(O, E, w=None, gamma=1j, eps_pinv=0.0, soft=True, eps_snr=0.0, shift=0.0,
             n_eff=None):
    """thetadot = -gamma S^+ F for the sample set (O [n][P], E [n], weights w or uniform)."""
    S, F, Em, Ob, f, w = tdvp_matrices(O, E, w)
    if shift:
        S = S + shift * np.diag(np.diag(S).real)
    lam, V = np.linalg.eigh(S)
    rho = V.conj().T @ F
    rho_var = None
    if eps_snr > 0:
        rho_s = f @ V.conj()                      # rho_k(s) = sum_l conj(V_lk) f_l(s)
        rho_var = w @ np.abs(rho_s - rho[None, :]) ** 2
        if n_eff is None:
            n_eff = O.shape[0]
    lp = damping(lam, rho, rho_var, n_eff, eps_pinv, soft, eps_snr)
    thetadot = -gamma * (V @ (lp * rho))
    return thetadot, {"S": S, "F": F, "E": Em, "lam": lam, "V": V, "rho": rho,
                      "rho_var": rho_var, "lam_plus": lp}


def exact_tdvp_rhs(model, Lx, Ly, J, h, M, params, gamma=1j, eps_pinv=0.0, soft=True,
                   shift=0.0, sz0=False):
    """tdvp_rhs with exact sums over all basis states (the ExactSampler): weights p(s)."""
    N = Lx * Ly
    s = all_states(N, sz0)
    lp = logpsi(N, M, params, s)
    p = born_weights(lp)
    e = eloc(model, Lx, Ly, J, h, M, params, s)
    O = ok(N, M, params, s)
    return tdvp_rhs(O, e, p, gamma, eps_pinv, soft, 0.0, shift)


def fisher_norm(v, S):
    """||v||_S = (1/N_p) sqrt(v^H S v), N_p the number of components of v (section
    "Utilities", Stepper)."""
    v = np.asarray(v, np.complex128)
    return float(np.sqrt(max(0.0, (v.conj() @ S @ v).real))) / v.size


def adaptive_heun_step(f, y, t, tau, eps, norm, tau_max=np.inf, max_retries=50):
    """One accepted step of the adaptive second-order (Heun) integrator (section
    "Utilities", Stepper): a step of size tau and two of size tau/2 from (y, t), the
    difference delta = norm(y_tau - y_tau/2) measured with norm(v, info) where info is
    what f returned at (y, t), and the step size updated as tau <- tau (eps/delta)^(1/3).
    The step is accepted when delta <= eps (the two-half-step solution is kept), otherwise
    it is repeated with the updated tau.  f(y, t) -> (ydot, info).
    Returns (y_new, t_new, tau_next, tau_used, delta, retries)."""
    k1, info = f(y, t)
    for retry in range(max_retries + 1):
        k2 = f(y + tau * k1, t + tau)[0]
        y_full = y + 0.5 * tau * (k1 + k2)
        h1 = f(y + 0.5 * tau * k1, t + 0.5 * tau)[0]
        yh = y + 0.25 * tau * (k1 + h1)
        g1 = f(yh, t + 0.5 * tau)[0]
        g2 = f(yh + 0.5 * tau * g1, t + tau)[0]
        y_half = yh + 0.25 * tau * (g1 + g2)
        delta = norm(y_full - y_half, info)
        tau_new = tau_max if delta == 0 else tau * (eps / delta) ** (1.0 / 3.0)
        tau_new = min(tau_new, tau_max)
        if delta <= eps:
            return y_half, t + tau, tau_new, tau, delta, retry
        tau = tau_new
    raise RuntimeError("adaptive Heun: no accepted step within max_retries")
