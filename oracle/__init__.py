"""FP64 CPU oracle for one NQS variational Monte Carlo step (arXiv:2108.03409, jVMC).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct definitions that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.  It shares no code with
the CUDA path and never imports it.

The arithmetic lives in ``vmc_oracle.c`` (compiled by :func:`build` with gcc/OpenMP);
this module marshals numpy arrays and adds the pieces that are naturally written with
numpy: exact enumeration of the Hilbert space (the paper's ExactSampler, section
"Sampler") and the integrated autocorrelation time.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  logpsi          -- pinned: brute-force sum over hidden units, W = 0 closed form
  connected/eloc  -- pinned: dense-H matvec by exact enumeration, Sx worked example,
                     product-state closed form, eigenstate invariant
  ok              -- pinned: central finite differences (real and imaginary steps)
  sr_matrices     -- pinned: exact-energy finite-difference gradient (F), fidelity
                     expansion (S), Hermitian PSD, Sz = 0 null mode
  cholesky_solve  -- pinned: residual and numpy.linalg.solve
  sr_apply        -- pinned: equals shift(sr_matrices S) v formed densely
  cg_solve        -- pinned: agrees with the dense solve, residual
  metropolis      -- pinned: chi-square of the histogram against exact |psi|^2
  philox4x64      -- pinned: numpy.random.Philox bit-for-bit
  tau_int         -- pinned: AR(1) closed form
  made_forward    -- pinned: autoregressive property (flip tests), sum_s q(s) = 1 by
                     enumeration, brute-force conditionals
  made_grad       -- pinned: central finite differences of the loss
  adam_step       -- pinned: closed form of the first two steps
  made_sample     -- pinned: chi-square of the sample histogram against q
  tdvp.*          -- regularised TDVP right-hand side and adaptive Heun integrator
                     (oracle/tdvp.py); pinned in tests/test_oracle_tdvp_pins.py
  excited.*       -- excited-state search by projection (oracle/excited.py); pinned in
                     tests/test_oracle_excited_pins.py
  ar.*            -- the autoregressive network as the ansatz (oracle/ar.py); pinned in
                     tests/test_oracle_ar_pins.py
  cnn.*           -- the translation-symmetric CNN-ELU ansatz (oracle/cnn.py); pinned in
                     tests/test_oracle_cnn_pins.py
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODEL_TFIM = 0
MODEL_HEIS = 1

_lib = None


def build(force: bool = False) -> str:
    """Compile vmc_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-std=gnu11", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "orc_num_threads": (i32, []),
            "orc_set_num_threads": (None, [i32]),
            "orc_philox4x64": (i32, [P, P, P]),
            "orc_bonds": (i32, [i32, i32, P, P]),
            "orc_theta": (i32, [i32, i32, P, P, i64, P]),
            "orc_logpsi": (i32, [i32, i32, P, P, i64, P]),
            "orc_connected": (i32, [i32, i32, i32, f64, f64, P, P, P]),
            "orc_max_connected": (i32, [i32, i32, i32]),
            "orc_eloc": (i32, [i32, i32, i32, f64, f64, i32, P, P, i64, P]),
            "orc_ok": (i32, [i32, i32, P, P, i64, P]),
            "orc_sr_matrices": (i32, [i64, i64, P, P, P, P, P]),
            "orc_sr_entries": (i32, [i64, i64, P, P, i64, P, P, P, i64, P, P]),
            "orc_shift": (i32, [i64, P, f64, i32]),
            "orc_cholesky_solve": (i32, [i64, P, P, P]),
            "orc_cg_solve": (i32, [i64, i64, P, P, f64, i32, f64, i32, P, P, P]),
            "orc_sr_apply": (i32, [i64, i64, P, f64, i32, P, P]),
            "orc_update": (i32, [i64, P, P, f64]),
            "orc_metropolis": (i32, [i32, i32, i32, i32, P, i64, P, u64, u64, u64, u64, i32, i32,
                                     P, P, P]),
            "orc_made_nparams": (i64, [i32, i32]),
            "orc_made_forward": (i32, [i32, i32, P, P, i64, P, P]),
            "orc_made_grad": (i32, [i32, i32, P, P, i64, P, P]),
            "orc_adam_step": (i32, [i64, P, P, P, P, i32, f64, f64, f64, f64]),
            "orc_made_sample": (i32, [i32, i32, P, i64, u64, u64, u64, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def _cplx(params: np.ndarray) -> np.ndarray:
    """complex128 view -> contiguous float64 [.., 2] buffer."""
    p = np.ascontiguousarray(params, dtype=np.complex128)
    return p.view(np.float64)


def _spins(spins: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(spins, dtype=np.int8)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def n_params(N: int, M: int) -> int:
    return N + M + N * M


# ----------------------------------------------------------------------------------------
# RNG
# ----------------------------------------------------------------------------------------
def philox4x64(ctr, key) -> np.ndarray:
    """Philox4x64-10 block for one counter (4 x u64) and key (2 x u64)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, dtype=np.uint64)
    _check(_load().orc_philox4x64(_ptr(c), _ptr(k), _ptr(out)), "philox4x64")
    return out


# ----------------------------------------------------------------------------------------
# Lattice / Hamiltonian
# ----------------------------------------------------------------------------------------
def bonds(Lx: int, Ly: int):
    nb = 2 * Lx * Ly if Ly > 1 else Lx * Ly
    bi = np.zeros(nb, dtype=np.int32)
    bj = np.zeros(nb, dtype=np.int32)
    got = _load().orc_bonds(Lx, Ly, _ptr(bi), _ptr(bj))
    assert got == nb
    return bi, bj


def connected(model: int, Lx: int, Ly: int, J: float, h: float, s: np.ndarray):
    """Connected configurations s' and matrix elements H_ss' of one configuration
    (entry 0 is the diagonal); the get_s_primes interface for a single s."""
    N = Lx * Ly
    lib = _load()
    mc = lib.orc_max_connected(model, Lx, Ly)
    sp = np.zeros((mc, N), dtype=np.int8)
    el = np.zeros(mc, dtype=np.float64)
    s = _spins(s).reshape(N)
    cnt = lib.orc_connected(model, Lx, Ly, float(J), float(h), _ptr(s), _ptr(sp), _ptr(el))
    if cnt < 0:
        raise OracleError("connected failed")
    return sp[:cnt].copy(), el[:cnt].copy()


# ----------------------------------------------------------------------------------------
# RBM quantities
# ----------------------------------------------------------------------------------------
def theta(N: int, M: int, params: np.ndarray, spins: np.ndarray) -> np.ndarray:
    """theta_j = b_j + sum_i W_ji s_i (Eq. rbm_ex) of each configuration, [n][M] complex."""
    s = _spins(spins).reshape(-1, N)
    p = _cplx(params)
    out = np.zeros((s.shape[0], M, 2), dtype=np.float64)
    _check(_load().orc_theta(N, M, _ptr(p), _ptr(s), s.shape[0], _ptr(out)), "theta")
    return out[..., 0] + 1j * out[..., 1]


def logpsi(N: int, M: int, params: np.ndarray, spins: np.ndarray) -> np.ndarray:
    s = _spins(spins).reshape(-1, N)
    p = _cplx(params)
    out = np.zeros((s.shape[0], 2), dtype=np.float64)
    _check(_load().orc_logpsi(N, M, _ptr(p), _ptr(s), s.shape[0], _ptr(out)), "logpsi")
    return out[:, 0] + 1j * out[:, 1]


def eloc(model: int, Lx: int, Ly: int, J: float, h: float, M: int, params: np.ndarray,
         spins: np.ndarray) -> np.ndarray:
    N = Lx * Ly
    s = _spins(spins).reshape(-1, N)
    p = _cplx(params)
    out = np.zeros((s.shape[0], 2), dtype=np.float64)
    _check(_load().orc_eloc(model, Lx, Ly, float(J), float(h), M, _ptr(p), _ptr(s), s.shape[0],
                            _ptr(out)), "eloc")
    return out[:, 0] + 1j * out[:, 1]


def ok(N: int, M: int, params: np.ndarray, spins: np.ndarray) -> np.ndarray:
    s = _spins(spins).reshape(-1, N)
    p = _cplx(params)
    P = n_params(N, M)
    out = np.zeros((s.shape[0], P, 2), dtype=np.float64)
    _check(_load().orc_ok(N, M, _ptr(p), _ptr(s), s.shape[0], _ptr(out)), "ok")
    return out[..., 0] + 1j * out[..., 1]


def sr_matrices(O: np.ndarray, E: np.ndarray, want_S: bool = True):
    """S (P x P), F (P), <E> from per-sample O (Ns x P) and E_loc (Ns)."""
    O = np.ascontiguousarray(O, dtype=np.complex128)
    E = np.ascontiguousarray(E, dtype=np.complex128)
    Ns, P = O.shape
    S = np.zeros((P, P), dtype=np.complex128) if want_S else None
    F = np.zeros(P, dtype=np.complex128)
    Em = np.zeros(2, dtype=np.float64)
    _check(_load().orc_sr_matrices(Ns, P, _ptr(O.view(np.float64)), _ptr(E.view(np.float64)),
                                   None if S is None else _ptr(S.view(np.float64)),
                                   _ptr(F.view(np.float64)), _ptr(Em)), "sr_matrices")
    return S, F, Em[0] + 1j * Em[1]


def sr_entries(O: np.ndarray, E: np.ndarray, kk, ll, fk):
    """Selected S_{k,l} and F_k without forming S."""
    O = np.ascontiguousarray(O, dtype=np.complex128)
    E = np.ascontiguousarray(E, dtype=np.complex128)
    Ns, P = O.shape
    kk = np.ascontiguousarray(kk, dtype=np.int64)
    ll = np.ascontiguousarray(ll, dtype=np.int64)
    fk = np.ascontiguousarray(fk, dtype=np.int64)
    s_out = np.zeros(len(kk), dtype=np.complex128)
    f_out = np.zeros(len(fk), dtype=np.complex128)
    _check(_load().orc_sr_entries(Ns, P, _ptr(O.view(np.float64)), _ptr(E.view(np.float64)),
                                  len(kk), _ptr(kk), _ptr(ll), _ptr(s_out.view(np.float64)),
                                  len(fk), _ptr(fk), _ptr(f_out.view(np.float64))), "sr_entries")
    return s_out, f_out


def shift(S: np.ndarray, nu: float, mode: int = 0) -> np.ndarray:
    S = np.array(S, dtype=np.complex128, order="C", copy=True)
    _check(_load().orc_shift(S.shape[0], _ptr(S.view(np.float64)), float(nu), int(mode)), "shift")
    return S


def cholesky_solve(S: np.ndarray, F: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.complex128)
    F = np.ascontiguousarray(F, dtype=np.complex128)
    x = np.zeros_like(F)
    _check(_load().orc_cholesky_solve(S.shape[0], _ptr(S.view(np.float64)),
                                      _ptr(F.view(np.float64)), _ptr(x.view(np.float64))),
           "cholesky_solve")
    return x


def sr_apply(O: np.ndarray, v: np.ndarray, nu: float, mode: int = 0) -> np.ndarray:
    """S~ v = (1/Ns) Obar^H (Obar v) + D v without forming S (D = nu diag(S), or nu)."""
    O = np.ascontiguousarray(O, dtype=np.complex128)
    v = np.ascontiguousarray(v, dtype=np.complex128)
    Ns, P = O.shape
    y = np.zeros(P, dtype=np.complex128)
    _check(_load().orc_sr_apply(Ns, P, _ptr(O.view(np.float64)), float(nu), int(mode),
                                _ptr(v.view(np.float64)), _ptr(y.view(np.float64))), "sr_apply")
    return y


def cg_solve(O: np.ndarray, F: np.ndarray, nu: float, mode: int = 0, tol: float = 1e-10,
             maxit: int = 1000):
    O = np.ascontiguousarray(O, dtype=np.complex128)
    F = np.ascontiguousarray(F, dtype=np.complex128)
    Ns, P = O.shape
    x = np.zeros(P, dtype=np.complex128)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    _check(_load().orc_cg_solve(Ns, P, _ptr(O.view(np.float64)), _ptr(F.view(np.float64)),
                                float(nu), int(mode), float(tol), int(maxit),
                                _ptr(x.view(np.float64)), ctypes.addressof(it),
                                ctypes.addressof(rr)), "cg_solve")
    return x, it.value, rr.value


def update(params: np.ndarray, x: np.ndarray, dt: float) -> np.ndarray:
    p = np.array(params, dtype=np.complex128, copy=True)
    xx = np.ascontiguousarray(x, dtype=np.complex128)
    _check(_load().orc_update(p.shape[0], _ptr(p.view(np.float64)), _ptr(xx.view(np.float64)),
                              float(dt)), "update")
    return p


def metropolis(model: int, Lx: int, Ly: int, M: int, params: np.ndarray, spins: np.ndarray,
               seed: int, stream: int = 0, chain0: int = 0, sweep0: int = 0,
               n_sweeps: int = 1, sweep_len: int = 0, record: bool = False):
    """Run n_sweeps Metropolis sweeps on every chain.  Returns (final spins, recorded
    states [n_sweeps][C][N] or None, min decision margin per chain, accepts per chain)."""
    N = Lx * Ly
    s = np.array(_spins(spins).reshape(-1, N), copy=True)
    C = s.shape[0]
    p = _cplx(params)
    rec = np.zeros((n_sweeps, C, N), dtype=np.int8) if record else None
    mm = np.zeros(C, dtype=np.float64)
    acc = np.zeros(C, dtype=np.int64)
    _check(_load().orc_metropolis(model, Lx, Ly, M, _ptr(p), C, _ptr(s), int(seed), int(stream),
                                  int(chain0), int(sweep0), int(n_sweeps), int(sweep_len),
                                  _ptr(rec), _ptr(mm), _ptr(acc)), "metropolis")
    return s, rec, mm, acc


# ----------------------------------------------------------------------------------------
# Exact enumeration (the ExactSampler of the "Sampler" section): all basis states, or the
# Sz = 0 sector, with exact Born weights p = |psi|^2 / sum |psi|^2 (Eq. expectation_value).
# ----------------------------------------------------------------------------------------
def all_states(N: int, sz0: bool = False) -> np.ndarray:
    idx = np.arange(1 << N, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(N, dtype=np.int64)[None, :]) & 1
    s = (1 - 2 * bits).astype(np.int8)          # bit 0 <-> s = +1
    if sz0:
        s = s[s.sum(axis=1) == 0]
    return s


def born_weights(lp: np.ndarray) -> np.ndarray:
    w = np.exp(2.0 * (lp.real - lp.real.max()))
    return w / w.sum()


def exact_energy(model: int, Lx: int, Ly: int, J: float, h: float, M: int, params: np.ndarray,
                 sz0: bool = False):
    """<H> = sum_s p(s) E_loc(s) over the enumerated space (Eq. expectation_value)."""
    N = Lx * Ly
    s = all_states(N, sz0)
    lp = logpsi(N, M, params, s)
    p = born_weights(lp)
    e = eloc(model, Lx, Ly, J, h, M, params, s)
    return complex(np.sum(p * e)), s, p, e


def exact_sr(model: int, Lx: int, Ly: int, J: float, h: float, M: int, params: np.ndarray,
             sz0: bool = False):
    """S, F and <E> with exact Born weights instead of Monte Carlo means (Eq. qfm,
    Eq. force_vector with <.> = sum_s p(s) .)."""
    N = Lx * Ly
    E, s, p, e = exact_energy(model, Lx, Ly, J, h, M, params, sz0)
    O = ok(N, M, params, s)
    mo = p @ O
    Ob = O - mo[None, :]
    S = (Ob.conj().T * p[None, :]) @ Ob
    F = Ob.conj().T @ (p * (e - E))
    return S, F, E


# ----------------------------------------------------------------------------------------
# Integrated autocorrelation time with Sokal's automatic window (c = 5).
# ----------------------------------------------------------------------------------------
def tau_int(x: np.ndarray, c: float = 5.0) -> float:
    """tau_int = 1/2 + sum_{t=1}^{W} rho(t), W the smallest window with W >= c tau_int(W)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    d = x - x.mean()
    var = np.dot(d, d) / n
    if n < 4 or var == 0.0:
        return 0.5
    tau = 0.5
    for t in range(1, n):
        rho = np.dot(d[:-t], d[t:]) / (n * var)
        tau += rho
        if t >= c * tau:
            break
    return float(max(tau, 0.5))


def tau_int_chains(series: np.ndarray, c: float = 5.0) -> float:
    """Average tau_int over chains; series is [T][C]."""
    series = np.asarray(series, dtype=np.float64)
    return float(np.mean([tau_int(series[:, k], c) for k in range(series.shape[1])]))


# ----------------------------------------------------------------------------------------
# MADE proposal
# ----------------------------------------------------------------------------------------
def made_nparams(N: int, H: int) -> int:
    return int(_load().orc_made_nparams(N, H))


def made_forward(N: int, H: int, params: np.ndarray, spins: np.ndarray, want_z: bool = False):
    s = _spins(spins).reshape(-1, N)
    p = np.ascontiguousarray(params, dtype=np.float64)
    lq = np.zeros(s.shape[0])
    z = np.zeros((s.shape[0], N)) if want_z else None
    _check(_load().orc_made_forward(N, H, _ptr(p), _ptr(s), s.shape[0], _ptr(lq), _ptr(z)),
           "made_forward")
    return (lq, z) if want_z else lq


def made_grad(N: int, H: int, params: np.ndarray, spins: np.ndarray):
    s = _spins(spins).reshape(-1, N)
    p = np.ascontiguousarray(params, dtype=np.float64)
    g = np.zeros_like(p)
    L = ctypes.c_double(0.0)
    _check(_load().orc_made_grad(N, H, _ptr(p), _ptr(s), s.shape[0], _ptr(g),
                                 ctypes.addressof(L)), "made_grad")
    return g, L.value


def adam_step(theta, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    th = np.array(theta, dtype=np.float64, copy=True)
    mm = np.array(m, dtype=np.float64, copy=True)
    vv = np.array(v, dtype=np.float64, copy=True)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    _check(_load().orc_adam_step(th.size, _ptr(th), _ptr(mm), _ptr(vv), _ptr(gg), int(t),
                                 float(lr), float(b1), float(b2), float(eps)), "adam_step")
    return th, mm, vv


def made_sample(N: int, H: int, params: np.ndarray, n: int, seed: int, stream: int = 0,
                round_: int = 0):
    p = np.ascontiguousarray(params, dtype=np.float64)
    s = np.zeros((n, N), dtype=np.int8)
    lq = np.zeros(n)
    mm = np.zeros(n)
    _check(_load().orc_made_sample(N, H, _ptr(p), n, int(seed), int(stream), int(round_),
                                   _ptr(s), _ptr(lq), _ptr(mm)), "made_sample")
    return s, lq, mm
