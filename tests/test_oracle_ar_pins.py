"""Pins of the autoregressive-ansatz oracle (oracle/ar.py): psi = q^(1/2) with the masked
autoregressive network, checked against a dense Hamiltonian built independently, finite
differences, and the Jordan-Wigner ground energy reached by exact-enumeration SR."""
import numpy as np

import oracle
from oracle import ar
from paper_2108_03409_b300 import inputs

from test_oracle_pins import _dense_h, jordan_wigner_e0

T, HEIS = inputs.MODEL_TFIM, inputs.MODEL_HEIS


def test_local_energy_is_h_psi_over_psi():
    """E_loc(s) = (H psi)(s) / psi(s) with psi = q^(1/2) over all states (TFIM chain and the
    Heisenberg 4 x 2 lattice), and <H> = sum_s q(s) E_loc(s) = psi^T H psi."""
    for model, Lx, Ly, J, h in ((T, 8, 1, 1.0, 0.7), (HEIS, 4, 2, 1.0, 0.0)):
        N, Hh = Lx * Ly, 32
        p = inputs.made_params(N, Hh, seed=3, scale=1.3).astype(np.float64)
        s = oracle.all_states(N)
        psi = np.exp(ar.ar_logpsi(N, Hh, p, s))
        Hm = _dense_h(model, Lx, Ly, J, h)
        ref = (Hm @ psi) / psi
        got = ar.ar_eloc(model, Lx, Ly, J, h, Hh, p, s)
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
        E, _, q = ar.ar_exact_energy(model, Lx, Ly, J, h, Hh, p)
        assert abs(np.sum(q) - 1.0) <= 1e-12
        assert abs(E - psi @ (Hm @ psi)) <= 1e-10 * abs(E)


def test_log_derivatives_are_half_dlogq():
    """O_k = d log psi / d theta_k: central differences of (1/2) log q in every free
    parameter (masked ones have O = 0 exactly)."""
    N, Hh = 6, 32
    p = inputs.made_params(N, Hh, seed=4, scale=1.2).astype(np.float64)
    s = oracle.all_states(N)[::5]
    O = ar.ar_ok(N, Hh, p, s)
    eps = 1e-6
    rng = np.random.default_rng(0)
    for k in rng.choice(p.size, 60, replace=False):
        dp = np.zeros_like(p)
        dp[k] = eps
        fd = (ar.ar_logpsi(N, Hh, p + dp, s) - ar.ar_logpsi(N, Hh, p - dp, s)) / (2 * eps)
        assert np.max(np.abs(fd - O[:, k])) <= 1e-7 * max(1.0, np.max(np.abs(O[:, k])))


def test_exact_sr_reaches_jordan_wigner():
    """Exact-enumeration SR of the autoregressive ansatz (N = 8 chain, J = h = 1, H = 32,
    dt 0.05, additive shift 1e-3 -- masked and inactive weights have zero rows in S, which a
    multiplicative shift leaves singular) reaches 1e-3 of the Jordan-Wigner energy within
    60 steps."""
    N, Hh, J, h = 8, 32, 1.0, 1.0
    E0 = jordan_wigner_e0(N, J, h)
    p = inputs.made_params(N, Hh, seed=5).astype(np.float64)
    s = oracle.all_states(N)
    for step in range(60):
        q = np.exp(oracle.made_forward(N, Hh, p, s))
        E = ar.ar_eloc(T, N, 1, J, h, Hh, p, s)
        O = ar.ar_ok(N, Hh, p, s)
        p, Em = ar.ar_sr_update(O, E, p, 0.05, 1e-3, mode=1, weights=q)
        if abs(Em - E0) / abs(E0) <= 1e-3:
            break
    assert abs(Em - E0) / abs(E0) <= 1e-3, (step, Em, E0)
