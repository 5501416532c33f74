"""FP64 oracle of the translation-symmetric single-layer CNN ansatz with ELU activation
(arXiv:2108.03409, section "Ground state search", Eq. gs_nqs):
    log psi(s) = sum_{a=1}^{alpha} sum_{omega in T} f_ELU(sum_l W_al s_omega(l) + b_a),
f_ELU(x) = x (x > 0), e^x - 1 (x <= 0), T the N translations of the periodic chain,
s_omega_r(l) = s_{(l + r) mod N}.  Real parameters [W (alpha x N, row-major) | b (alpha)],
real log psi (positive amplitudes, the TFIM ground state's sign structure).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  Plain numpy definitions:
    z_ar(s)   = sum_l W_al s_{(l+r) mod N} + b_a,
    O_{W_al}  = sum_r f'(z_ar) s_{(l+r) mod N},  O_{b_a} = sum_r f'(z_ar),  f'(x) = 1 or e^x,
    E_loc(s)  = sum_s' H_ss' psi(s')/psi(s)    (psi(s') evaluated from scratch),
and single-flip Metropolis with the same Philox4x64-10 stream and acceptance rule as the
RBM sampler (counter {chain, sweep, step, 0}, key {seed, stream}; site floor((w0 >> 32) N
/ 2^32), u = ((w1 >> 40) + 1/2) / 2^24, accept iff ln u < 2 (log psi(s') - log psi(s))).

Parity status: pinned in tests/test_oracle_cnn_pins.py (translation invariance, central
finite differences, dense-H local energy, exact SR reaching the Jordan-Wigner energy, and
the Metropolis chain's stationary histogram).
"""
from __future__ import annotations

import numpy as np

from . import connected, philox4x64


def nparams(N: int, alpha: int) -> int:
    return alpha * (N + 1)


def _split(params, N, alpha):
    p = np.asarray(params, np.float64)
    return p[:alpha * N].reshape(alpha, N), p[alpha * N:alpha * N + alpha]


def _shifted(spins, N):
    s = np.asarray(spins, np.float64).reshape(-1, N)
    idx = (np.arange(N)[None, :] + np.arange(N)[:, None]) % N     # [r][l] -> (l + r) mod N
    return s[:, idx]                                               # [n][r][l]


def preact(N, alpha, params, spins):
    W, b = _split(params, N, alpha)
    return np.einsum("nrl,al->nar", _shifted(spins, N), W) + b[None, :, None]


def elu(x):
    return np.where(x > 0, x, np.expm1(np.minimum(x, 0.0)))


def logpsi(N, alpha, params, spins):
    return elu(preact(N, alpha, params, spins)).sum(axis=(1, 2))


def ok(N, alpha, params, spins):
    z = preact(N, alpha, params, spins)
    d = np.where(z > 0, 1.0, np.exp(np.minimum(z, 0.0)))          # f'(z)
    OW = np.einsum("nar,nrl->nal", d, _shifted(spins, N))
    Ob = d.sum(axis=2)
    return np.concatenate([OW.reshape(len(z), -1), Ob], axis=1)


def eloc(model, Lx, Ly, J, h, alpha, params, spins):
    N = Lx * Ly
    s = np.asarray(spins, np.int8).reshape(-1, N)
    out = np.zeros(len(s))
    for q, c in enumerate(s):
        sp, el = connected(model, Lx, Ly, J, h, c)
        lp = logpsi(N, alpha, params, sp)
        out[q] = np.sum(el * np.exp(lp - lp[0]))
    return out


def metropolis(N, alpha, params, spins, seed, stream=0, sweep0=0, n_sweeps=1, record=False):
    """Single-flip Metropolis of every chain; returns (final, records [n_sweeps][C][N] or
    None, min decision margin per chain).  The chains advance in lock-step (one step of
    every chain, then the next), each with its own counter-based draws."""
    s = np.array(spins, np.int8).reshape(-1, N)
    C = len(s)
    lp = logpsi(N, alpha, params, s)
    rec = np.zeros((n_sweeps, C, N), np.int8) if record else None
    margin = np.full(C, np.inf)
    rows = np.arange(C)
    for k in range(n_sweeps):
        for t in range(N):
            w = np.array([philox4x64([c, sweep0 + k, t, 0], [seed, stream]) for c in range(C)])
            site = ((w[:, 0] >> np.uint64(32)) * np.uint64(N)) >> np.uint64(32)
            u = ((w[:, 1] >> np.uint64(40)).astype(np.float64) + 0.5) / 2.0 ** 24
            sp = s.copy()
            sp[rows, site.astype(np.int64)] *= -1
            lpp = logpsi(N, alpha, params, sp)
            d = 2.0 * (lpp - lp)
            margin = np.minimum(margin, np.abs(np.log(u) - d))
            acc = np.log(u) < d
            s[acc] = sp[acc]
            lp[acc] = lpp[acc]
        if record:
            rec[k] = s
    return s, rec, margin
