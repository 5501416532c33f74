"""Seeded synthetic inputs for the NQS-VMC hot path.

This module holds no arithmetic of the method itself: it only draws random parameters,
spin configurations and couplings from fixed seeds and describes the workload sizes.
Both the CUDA path and the CPU oracle receive what it produces, so initialisation is
never a parity question.

Recipes (numpy PCG64 generators, one per seed):
  * RBM parameters: Re and Im of every complex parameter drawn independently from
    N(0, sigma^2); optional Marshall phase: a_i += i*pi/2 on the sublattice (x + y) even,
    which makes exp(sum_i a_i s_i) carry the Marshall sign (-1)^{N_up on A} up to a
    global phase.
  * Chains: uniform +-1 spins (TFIM), or a uniformly random arrangement of N/2 up and
    N/2 down spins (Heisenberg, Sz = 0 sector).
  * Batched TFIM fields: h_l ~ U[2, 4] (J = 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

MODEL_TFIM = 0
MODEL_HEIS = 1


def n_params(N: int, M: int) -> int:
    """P = N + M + N*M complex parameters, ordered [a(N) | b(M) | W(M x N row-major)]."""
    return N + M + N * M


def rbm_params(N: int, M: int, sigma: float, seed: int,
               marshall: Optional[Tuple[int, int]] = None) -> np.ndarray:
    """Complex parameter vector (complex128, length P)."""
    rng = np.random.default_rng(seed)
    P = n_params(N, M)
    re = rng.normal(0.0, sigma, P)
    im = rng.normal(0.0, sigma, P)
    p = re + 1j * im
    if marshall is not None:
        Lx, Ly = marshall
        assert Lx * Ly == N
        for y in range(Ly):
            for x in range(Lx):
                if (x + y) % 2 == 0:
                    p[x + Lx * y] += 0.5j * np.pi
    return p


def made_params(N: int, H: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Initial parameters of the learned proposal, float32, layout W1[H][N] | b1[H] |
    W2[H][H] | b2[H] | W3[N][H] | b3[N]: weights N(0, scale^2 / fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, scale / np.sqrt(N), (H, N))
    W2 = rng.normal(0.0, scale / np.sqrt(H), (H, H))
    W3 = rng.normal(0.0, scale / np.sqrt(H), (N, H))
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3.ravel(),
                           np.zeros(N)]).astype(np.float32)


def random_spins(C: int, N: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (1 - 2 * rng.integers(0, 2, size=(C, N))).astype(np.int8)


def random_sz0_spins(C: int, N: int, seed: int) -> np.ndarray:
    assert N % 2 == 0
    rng = np.random.default_rng(seed)
    base = np.concatenate([np.ones(N // 2, np.int8), -np.ones(N // 2, np.int8)])
    out = np.empty((C, N), dtype=np.int8)
    for c in range(C):
        out[c] = rng.permutation(base)
    return out


def initial_spins(model: int, C: int, N: int, seed: int) -> np.ndarray:
    return random_sz0_spins(C, N, seed) if model == MODEL_HEIS else random_spins(C, N, seed)


def uniform_fields(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, n)


@dataclass
class Lattice:
    model: int
    Lx: int
    Ly: int
    J: float = 1.0
    h: float = 0.0
    alpha: int = 1

    @property
    def N(self) -> int:
        return self.Lx * self.Ly

    @property
    def M(self) -> int:
        return self.alpha * self.N

    @property
    def P(self) -> int:
        return n_params(self.N, self.M)


@dataclass
class Workload:
    """One synthetic workload: lattices, chains, sweeps, SR settings and seeds."""
    name: str
    lattices: List[Lattice]
    chains: int
    sweeps_per_step: int
    therm_sweeps: int
    sr_steps: int
    dt: float
    shift: float
    sigma: float = 0.01
    param_seed: int = 1234
    chain_seed: int = 99
    rng_seed: int = 1
    marshall: bool = False
    solver: str = "cholesky"
    extra: dict = field(default_factory=dict)


def tfim_chain_10() -> Workload:
    """1D TFIM N=10 PBC, J=h=1, alpha=1; 256 chains x 200 sweeps per SR step."""
    return Workload("tfim1d_N10_alpha1_c256", [Lattice(MODEL_TFIM, 10, 1, 1.0, 1.0, 1)],
                    chains=256, sweeps_per_step=200, therm_sweeps=20, sr_steps=50, dt=0.02,
                    shift=1e-4)


def heisenberg_8x8() -> Workload:
    """2D Heisenberg 8x8 PBC, Marshall phase, alpha=2 (M=128, P=8384); 8192 chains, one
    sample per chain per SR step (one exchange sweep apart), dense S, Cholesky solve."""
    return Workload("heis2d_8x8_alpha2_c8192", [Lattice(MODEL_HEIS, 8, 8, 1.0, 0.0, 2)],
                    chains=8192, sweeps_per_step=1, therm_sweeps=20, sr_steps=1, dt=0.02,
                    shift=1e-3, marshall=True)


def tfim_batched_48(seed: int = 7) -> Workload:
    """48 independent 2D TFIM lattices (16 each of 4x4, 6x6, 8x8), h ~ U[2,4], alpha=2,
    1024 chains per lattice."""
    hs = uniform_fields(48, 2.0, 4.0, seed)
    lats = []
    for k, L in enumerate([4] * 16 + [6] * 16 + [8] * 16):
        lats.append(Lattice(MODEL_TFIM, L, L, 1.0, float(hs[k]), 2))
    return Workload("tfim2d_batched48_alpha2_c1024", lats, chains=1024, sweeps_per_step=1,
                    therm_sweeps=20, sr_steps=1, dt=0.02, shift=1e-3)


def tfim_12x12() -> Workload:
    return Workload("tfim2d_12x12_h3.04_alpha2_c16384", [Lattice(MODEL_TFIM, 12, 12, 1.0, 3.04, 2)],
                    chains=16384, sweeps_per_step=1, therm_sweeps=20, sr_steps=1, dt=0.02,
                    shift=1e-3, solver="cg")


def heisenberg_16x16() -> Workload:
    return Workload("heis2d_16x16_alpha2_c65536", [Lattice(MODEL_HEIS, 16, 16, 1.0, 0.0, 2)],
                    chains=65536, sweeps_per_step=1, therm_sweeps=20, sr_steps=1, dt=0.02,
                    shift=1e-3, marshall=True, solver="cg")


def workload_params(w: Workload, lattice_index: int = 0) -> np.ndarray:
    lat = w.lattices[lattice_index]
    return rbm_params(lat.N, lat.M, w.sigma, w.param_seed + lattice_index,
                      (lat.Lx, lat.Ly) if w.marshall else None)


def workload_spins(w: Workload, lattice_index: int = 0) -> np.ndarray:
    lat = w.lattices[lattice_index]
    return initial_spins(lat.model, w.chains, lat.N, w.chain_seed + lattice_index)
