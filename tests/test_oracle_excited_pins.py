"""Pins of the excited-state oracle (oracle/excited.py): the projected ansatz
Psi = psi - lambda phi of the section "Finding low-energy states", checked against dense
amplitude vectors and a dense Hamiltonian built independently (bit operations), and the
search reaching the first excited energy of exact diagonalisation."""
import numpy as np

import oracle
from oracle import excited
from paper_2108_03409_b300 import inputs

from test_oracle_pins import _dense_h

T = inputs.MODEL_TFIM


def _amplitudes(N, M, p):
    s = oracle.all_states(N)
    return s, np.exp(oracle.logpsi(N, M, p, s))


def _pair(N, M, seed):
    return (inputs.rbm_params(N, M, 0.3, seed=seed), inputs.rbm_params(N, M, 0.3, seed=seed + 1))


def test_lambda_is_the_overlap_ratio():
    """<psi/phi> under |phi|^2 with exact sums equals <phi|psi> / <phi|phi> of the vectors."""
    N, M = 6, 6
    p_psi, p_phi = _pair(N, M, 3)
    _, a = _amplitudes(N, M, p_psi)
    _, b = _amplitudes(N, M, p_phi)
    ref = np.vdot(b, a) / np.vdot(b, b)
    lam = excited.overlap_ratio_exact(N, M, p_psi, p_phi)
    assert abs(lam - ref) <= 1e-12 * abs(ref)
    # and Psi = psi - lambda phi is orthogonal to phi
    assert abs(np.vdot(b, a - lam * b)) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)


def test_local_energy_and_weights_of_the_projected_ansatz():
    """E_loc^Psi(s) = (H Psi)(s) / Psi(s) with the dense H, and the importance-weighted
    average over |psi|^2 equals <Psi|H|Psi> / <Psi|Psi>."""
    N, M, J, h = 6, 6, 1.0, 0.7
    p_psi, p_phi = _pair(N, M, 5)
    s, a = _amplitudes(N, M, p_psi)
    _, b = _amplitudes(N, M, p_phi)
    lam = excited.overlap_ratio_exact(N, M, p_psi, p_phi)
    Psi = a - lam * b
    H = _dense_h(T, N, 1, J, h)
    ref = (H @ Psi) / Psi
    rho, e, O, w = excited.excited_quantities(T, N, 1, J, h, M, p_psi, p_phi, lam, s)
    assert np.max(np.abs(e - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.allclose(w, np.abs(Psi / a) ** 2, rtol=1e-12)
    E, _ = excited.exact_excited_energy(T, N, 1, J, h, M, p_psi, p_phi)
    Eref = np.vdot(Psi, H @ Psi) / np.vdot(Psi, Psi)
    assert abs(E - Eref) <= 1e-12 * abs(Eref)


def test_log_derivatives_of_the_projected_ansatz():
    """O_k^Psi = d log Psi / d theta_k (phi fixed): central differences with real and
    imaginary steps (holomorphic)."""
    N, M = 4, 4
    p_psi, p_phi = _pair(N, M, 7)
    lam = 0.3 - 0.2j
    s = oracle.all_states(N)[::3]
    _, _, O, _ = excited.excited_quantities(T, N, 1, 1.0, 1.0, M, p_psi, p_phi, lam, s)

    def logPsi(p):
        return np.log(np.exp(oracle.logpsi(N, M, p, s)) - lam * np.exp(oracle.logpsi(N, M, p_phi, s)))

    eps = 1e-6
    for k in range(0, p_psi.size, 3):
        for step in (eps, 1j * eps):
            dp = np.zeros_like(p_psi)
            dp[k] = step
            fd = (logPsi(p_psi + dp) - logPsi(p_psi - dp)) / (2 * step)
            assert np.max(np.abs(fd - O[:, k])) <= 1e-7 * max(1.0, np.max(np.abs(O[:, k])))


def test_search_reaches_the_first_excited_energy():
    """Ground state by exact SR (120 steps), then the alternating search (exact lambda, one
    SR step of Psi with exact sums, dt 0.05, shift 1e-3) of the N = 8 chain at J = h = 1:
    within 120 steps <Psi|H|Psi>/<Psi|Psi> is within 1e-3 of E_1 from dense ED."""
    N, M, J, h = 8, 8, 1.0, 1.0
    ev = np.linalg.eigvalsh(_dense_h(T, N, 1, J, h).toarray())
    E1 = ev[1]
    p = inputs.rbm_params(N, M, 0.01, seed=1234)
    for _ in range(120):
        S, F, E = oracle.exact_sr(T, N, 1, J, h, M, p)
        p = oracle.update(p, oracle.cholesky_solve(oracle.shift(S, 1e-4, 0), F), 0.05)
    assert abs(E.real - ev[0]) <= 1e-3 * abs(ev[0])
    phi = p
    psi = inputs.rbm_params(N, M, 0.1, seed=77)
    s = oracle.all_states(N)
    for step in range(120):
        lam = excited.overlap_ratio_exact(N, M, psi, phi)
        pw = oracle.born_weights(oracle.logpsi(N, M, psi, s))
        td, info = excited.excited_rhs(T, N, 1, J, h, M, psi, phi, lam, s, psi_weights=pw,
                                       shift=1e-3)
        psi = psi + 0.05 * td
    E, _ = excited.exact_excited_energy(T, N, 1, J, h, M, psi, phi)
    assert abs(E.real - E1) <= 1e-3 * abs(E1), (E.real, E1)
    assert E.real >= ev[0]
