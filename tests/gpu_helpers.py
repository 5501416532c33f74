"""Shared helpers of the GPU parity tests (contexts, tolerances, comparisons)."""
import contextlib

import numpy as np

from paper_2108_03409_b300 import inputs
from paper_2108_03409_b300 import vmc

# Tolerances (FP32 path against the FP64 oracle):
LOGPSI_ABS = 1e-5          # |d log psi| at init-scale weights (phase compared mod 2 pi)
ELOC_PER_SITE_ABS = 1e-5   # |d E_loc| / N
OK_REL = 1e-5              # |d O_k| <= OK_REL * |O_k| + OK_ABS
OK_ABS = 1e-7
# S is a serial FP32 sum of n products per entry on the SIMT path: the worst-case
# relative error of such a sum is n * 2^-24 (stated relative to the largest diagonal
# element of S, which bounds every |S_kl| by Cauchy-Schwarz).
def s_tol_fp32(n):
    return n * 2.0 ** -24


# F is summed in FP32 over sub-chunks of 128 samples and in FP64 across them.
F_REL = 128 * 2.0 ** -24 * 4
# BF16 hi/lo split: each operand keeps ~16 bits, the dropped lo*lo term is 2^-16 relative
S_REL_BF16 = 1e-4


def torch_dev():
    import torch
    return torch


def lattice(model, Lx, Ly, J=1.0, h=1.0, alpha=1):
    return vmc.make_lattice(model, Lx, Ly, J, h, alpha)


@contextlib.contextmanager
def context(lat, **cfg):
    ctx = vmc.vmc_init(vmc.make_config(**cfg), [lat])
    try:
        yield ctx
    finally:
        vmc.vmc_destroy(ctx)


def phase_diff(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b))))


def to_dev_spins(s):
    import torch
    return torch.from_numpy(np.ascontiguousarray(s, dtype=np.int8)).cuda()


def cplx(t):
    a = t.cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def well_conditioned(p, s, N, M, cut=0.02):
    """Mask of configurations whose amplitude is not within `cut` of a node of psi:
    min_j |cosh theta_j| >= cut.  Near a node log psi and E_loc are ill-conditioned (an
    FP32 rounding of theta is amplified by |tanh theta_j|), so element-wise FP32 parity is
    only asserted away from them."""
    b = p[N:N + M]
    W = p[N + M:].reshape(M, N)
    theta = b[None, :] + s.astype(np.float64) @ W.T
    return np.min(np.abs(np.cosh(theta)), axis=1) >= cut


def eloc_tolerance(model, Lx, Ly, J, h, M, p, s):
    """Per-sample bound on |E_loc(GPU) - E_loc(oracle)|: ELOC_PER_SITE_ABS * N plus
    2e-5 times the sum of the magnitudes of the terms H_ss' psi(s')/psi(s).  Every term is
    an FP32 product whose relative error grows with |tanh theta| (near a node of psi the
    terms, and with them the error, become large); away from nodes the sum is O(N) and the
    bound reduces to the absolute per-site one."""
    import oracle
    N = Lx * Ly
    out = np.empty(len(s))
    for q, c in enumerate(s):
        sp, el = oracle.connected(model, Lx, Ly, J, h, c)
        lp = oracle.logpsi(N, M, p, sp)
        out[q] = np.sum(np.abs(el) * np.abs(np.exp(lp - lp[0])))
    return ELOC_PER_SITE_ABS * N + 2e-5 * out


def spins_for(model, C, N, seed):
    return inputs.initial_spins(model, C, N, seed)
