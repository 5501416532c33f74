"""FP64 oracle of the excited-state search by projection (arXiv:2108.03409, section
"Finding low-energy states", Eq. excited_state_ansatz and the overlap lambda after it).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

With a converged ground-state ansatz phi = psi_{theta*} the excited-state ansatz is
    Psi(s) = psi_theta(s) - lambda phi(s),   lambda = <phi|psi> / <phi|phi> = <psi / phi>_phi,
and one step of the search computes lambda (from samples of |phi|^2), then one SR step of
Psi.  Everything about Psi follows from the two RBMs and rho(s) = lambda phi(s) / psi(s):
    Psi(s) / psi(s) = 1 - rho(s),
    E_loc^Psi(s)    = (E_loc^psi(s) - rho(s) E_loc^phi(s)) / (1 - rho(s)),
    O_k^Psi(s)      = O_k^psi(s) / (1 - rho(s))       (phi does not depend on theta).
Reading (the paper does not say how |Psi|^2 is sampled): expectations under |Psi|^2 are
estimated from samples of |psi_theta|^2 with the importance weights |1 - rho(s)|^2, the
sampler of psi being reused unchanged.

Parity status: pinned in tests/test_oracle_excited_pins.py (lambda against the overlap of
the enumerated amplitude vectors, E_loc^Psi against a dense-H matvec, O^Psi against
finite differences of log Psi, the orthogonality <phi|Psi> = 0, the weighted estimator
against exact |Psi|^2 sums, and the search reaching the first excited energy of dense ED).
"""
from __future__ import annotations

import numpy as np

from . import all_states, born_weights, eloc, logpsi, ok
from . import tdvp as _tdvp


def overlap_ratio(N, M, p_psi, p_phi, spins_phi):
    """lambda = <psi / phi> over samples of |phi|^2 (uniform mean), complex."""
    d = logpsi(N, M, p_psi, spins_phi) - logpsi(N, M, p_phi, spins_phi)
    m = np.max(d.real)
    return np.exp(m) * np.mean(np.exp(d - m))


def overlap_ratio_exact(N, M, p_psi, p_phi):
    """lambda with exact sums: sum_s |phi|^2/Z_phi * psi/phi."""
    s = all_states(N)
    lf = logpsi(N, M, p_phi, s)
    w = born_weights(lf)
    d = logpsi(N, M, p_psi, s) - lf
    m = np.max(d.real)
    return np.exp(m) * np.sum(w * np.exp(d - m))


def excited_quantities(model, Lx, Ly, J, h, M, p_psi, p_phi, lam, spins):
    """Per configuration: rho, E_loc^Psi, O^Psi [n][P], importance weight |1 - rho|^2."""
    N = Lx * Ly
    lp = logpsi(N, M, p_psi, spins)
    lf = logpsi(N, M, p_phi, spins)
    rho = lam * np.exp(lf - lp)
    ep = eloc(model, Lx, Ly, J, h, M, p_psi, spins)
    ef = eloc(model, Lx, Ly, J, h, M, p_phi, spins)
    e = (ep - rho * ef) / (1.0 - rho)
    O = ok(N, M, p_psi, spins) / (1.0 - rho)[:, None]
    w = np.abs(1.0 - rho) ** 2
    return rho, e, O, w


def excited_rhs(model, Lx, Ly, J, h, M, p_psi, p_phi, lam, spins, psi_weights=None,
                shift=0.0, eps_pinv=0.0, soft=True):
    """SR direction thetadot = -S^+ F of Psi (gamma = 1) from configurations sampled from
    |psi|^2 (psi_weights None: Monte Carlo samples, uniform) or weighted by psi_weights
    (e.g. exact Born weights of psi), with the importance weights |1 - rho|^2."""
    rho, e, O, w = excited_quantities(model, Lx, Ly, J, h, M, p_psi, p_phi, lam, spins)
    if psi_weights is not None:
        w = w * psi_weights
    td, info = _tdvp.tdvp_rhs(O, e, w, gamma=1.0, eps_pinv=eps_pinv, soft=soft, shift=shift)
    info["rho"] = rho
    info["E_psi_exc"] = info["E"]
    return td, info


def exact_excited_energy(model, Lx, Ly, J, h, M, p_psi, p_phi, lam=None):
    """<Psi|H|Psi> / <Psi|Psi> by enumeration, with lambda exact unless given."""
    N = Lx * Ly
    if lam is None:
        lam = overlap_ratio_exact(N, M, p_psi, p_phi)
    s = all_states(N)
    pw = born_weights(logpsi(N, M, p_psi, s))
    rho, e, O, w = excited_quantities(model, Lx, Ly, J, h, M, p_psi, p_phi, lam, s)
    ww = pw * w
    return complex(np.sum(ww * e) / np.sum(ww)), lam
