"""FP64 oracle of the autoregressive neural quantum state used as the ansatz (arXiv:
2108.03409, section "Autoregressive neural quantum states"): psi(s) = q(s)^(1/2) with q the
masked autoregressive network of the MADE part of this oracle (normalised by construction,
sum_s q(s) = 1), sampled directly (one exact draw per sample, no Markov chain).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

The amplitudes are real and positive (real network parameters, no phase output): enough for
the stoquastic TFIM whose ground state is positive, which is the paper's autoregressive
example (a TFIM chain).  With real parameters the SR equation is real (Eq. tdvp_re with
gamma = 1: Re S and Re F, and here S and F are real already):
    O_k(s) = d log psi(s) / d theta_k = (1/2) d log q(s) / d theta_k,
    E_loc(s) = sum_s' H_ss' (q(s') / q(s))^(1/2),
    theta <- theta - dt (S + shift)^-1 F.

Parity status: pinned in tests/test_oracle_ar_pins.py (E_loc against a dense-H matvec on the
enumerated amplitude vector, O_k against central finite differences of log psi, <H> by
enumeration, and exact-enumeration SR lowering the energy towards the Jordan-Wigner value).
"""
from __future__ import annotations

import numpy as np

from . import all_states, cholesky_solve, connected, made_forward, made_grad, shift, sr_matrices


def ar_logpsi(N, H, params, spins):
    return 0.5 * made_forward(N, H, params, spins)


def ar_eloc(model, Lx, Ly, J, h, H, params, spins):
    N = Lx * Ly
    s = np.asarray(spins, np.int8).reshape(-1, N)
    out = np.zeros(len(s))
    for q, c in enumerate(s):
        sp, el = connected(model, Lx, Ly, J, h, c)
        lq = made_forward(N, H, params, sp)
        out[q] = np.sum(el * np.exp(0.5 * (lq - lq[0])))
    return out


def ar_ok(N, H, params, spins):
    """O [n][P] (real): per sample, -1/2 times the gradient of -log q(s)."""
    s = np.asarray(spins, np.int8).reshape(-1, N)
    return np.stack([-0.5 * made_grad(N, H, params, s[q:q + 1])[0] for q in range(len(s))])


def ar_sr_update(O, E, params, dt, nu, mode=0, weights=None):
    """One SR step from per-sample O, E (uniform weights, or exact weights w)."""
    if weights is None:
        S, F, Em = sr_matrices(O, E)
    else:
        w = np.asarray(weights, np.float64) / np.sum(weights)
        Em = np.sum(w * E)
        Ob = O - (w @ O)[None, :]
        S = (Ob.T * w[None, :]) @ Ob
        F = Ob.T @ (w * (E - Em))
    x = cholesky_solve(shift(np.asarray(S, np.complex128), nu, mode), np.asarray(F, np.complex128))
    return np.asarray(params, np.float64) - dt * x.real, Em


def ar_exact_energy(model, Lx, Ly, J, h, H, params):
    """<H> = sum_s q(s) E_loc(s) over all states (q is normalised)."""
    N = Lx * Ly
    s = all_states(N)
    q = np.exp(made_forward(N, H, params, s))
    return float(np.sum(q * ar_eloc(model, Lx, Ly, J, h, H, params, s))), s, q
