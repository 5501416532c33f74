"""Thin ctypes binding of libvmc (include/vmc.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors and
Python values into the C ABI's pointers and structs and turns status codes into
exceptions.  The function names are the C entry points.  The library is loaded on first
use; if ``libvmc.so`` is missing the call raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvmc.so")

VMC_OK, VMC_ERR_ARG, VMC_ERR_CUDA, VMC_ERR_OOM, VMC_ERR_NUMERIC, VMC_ERR_TIMEOUT, VMC_ERR_STATE = range(7)
MODEL_TFIM, MODEL_HEISENBERG = 0, 1
PREC_FP32, PREC_BF16SPLIT = 0, 1
SOLVER_CHOLESKY_FP64, SOLVER_CG, SOLVER_CHOLESKY_MIXED, SOLVER_CHOLESKY_TC = 0, 1, 2, 3
SHIFT_MULTIPLICATIVE, SHIFT_ADDITIVE = 0, 1

_STATUS_NAMES = {0: "VMC_OK", 1: "VMC_ERR_ARG", 2: "VMC_ERR_CUDA", 3: "VMC_ERR_OOM",
                 4: "VMC_ERR_NUMERIC", 5: "VMC_ERR_TIMEOUT", 6: "VMC_ERR_STATE"}


class VmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class vmc_lattice(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("Lx", ctypes.c_int), ("Ly", ctypes.c_int),
                ("J", ctypes.c_double), ("h", ctypes.c_double), ("alpha", ctypes.c_int)]


class vmc_config(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_chains", ctypes.c_int), ("sweep_len", ctypes.c_int),
                ("therm_sweeps", ctypes.c_int), ("sweeps_per_sample", ctypes.c_int),
                ("samples_per_chain", ctypes.c_int), ("precision", ctypes.c_int),
                ("solver", ctypes.c_int), ("shift", ctypes.c_double), ("shift_mode", ctypes.c_int),
                ("cg_maxit", ctypes.c_int), ("cg_tol", ctypes.c_double),
                ("made_hidden", ctypes.c_int), ("made_batch", ctypes.c_int),
                ("tdvp", ctypes.c_int), ("ar_ansatz", ctypes.c_int), ("cnn_ansatz", ctypes.c_int)]


class vmc_sr_stats(ctypes.Structure):
    _fields_ = [("e_mean_re", ctypes.c_double), ("e_mean_im", ctypes.c_double),
                ("e_var", ctypes.c_double), ("e_stderr", ctypes.c_double),
                ("acceptance", ctypes.c_double), ("n_samples", ctypes.c_int64),
                ("solver_iters", ctypes.c_int), ("solver_relres", ctypes.c_double),
                ("ms_sample", ctypes.c_float), ("ms_grad", ctypes.c_float),
                ("ms_qfm", ctypes.c_float), ("ms_solve", ctypes.c_float),
                ("ms_update", ctypes.c_float), ("ms_gram", ctypes.c_float),
                ("launches", ctypes.c_int64), ("solver_converged", ctypes.c_int),
                ("solver_relres_explicit", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vmc_tdvp_opts(ctypes.Structure):
    _fields_ = [("gamma_re", ctypes.c_double), ("gamma_im", ctypes.c_double),
                ("eps_pinv", ctypes.c_double), ("pinv_soft", ctypes.c_int),
                ("eps_snr", ctypes.c_double), ("shift", ctypes.c_double), ("exact", ctypes.c_int),
                ("eps_step", ctypes.c_double), ("tau_max", ctypes.c_double),
                ("max_retries", ctypes.c_int), ("jacobi_max_sweeps", ctypes.c_int)]


class vmc_tdvp_stats(ctypes.Structure):
    _fields_ = [("e_mean_re", ctypes.c_double), ("e_mean_im", ctypes.c_double),
                ("e_var", ctypes.c_double), ("e_stderr", ctypes.c_double),
                ("lam_max", ctypes.c_double), ("lam_min", ctypes.c_double), ("kept", ctypes.c_int),
                ("snr_min", ctypes.c_double), ("jacobi_sweeps", ctypes.c_int),
                ("jacobi_off", ctypes.c_double), ("tau_used", ctypes.c_double),
                ("tau_next", ctypes.c_double), ("delta", ctypes.c_double),
                ("retries", ctypes.c_int), ("rhs_evals", ctypes.c_int), ("ms", ctypes.c_float),
                ("ms_gram", ctypes.c_float), ("ms_eig", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vmc_excited_stats(ctypes.Structure):
    _fields_ = [("lambda_re", ctypes.c_double), ("lambda_im", ctypes.c_double),
                ("ess", ctypes.c_double), ("tdvp", vmc_tdvp_stats)]


EXPORTED = ["vmc_init", "vmc_destroy", "vmc_last_error", "vmc_set_params", "vmc_get_params",
            "vmc_set_chains", "vmc_get_chains", "vmc_theta", "vmc_logpsi", "vmc_local_energy", "vmc_sample",
            "vmc_grad", "vmc_qfm", "vmc_solve", "vmc_sr_step", "vmc_sr_step_on", "vmc_kernel_launches",
            "vmc_num_samples", "vmc_num_params", "vmc_force_noalloc", "vmc_cg_solve", "vmc_sr_apply",
            "vmc_made_set_params", "vmc_made_get_params", "vmc_made_logq", "vmc_made_grad",
            "vmc_proposal_train", "vmc_made_sample", "vmc_sample_learned", "vmc_sample_all",
            "vmc_autotuned_warps_per_block", "vmc_autotuned_slots_per_lane", "vmc_get_state", "vmc_set_state", "vmc_selftest_wait_timeout",
            "vmc_tdvp_rhs", "vmc_tdvp_step", "vmc_excited_lambda", "vmc_excited_rhs",
            "vmc_excited_step", "vmc_ar_set_params", "vmc_ar_get_params", "vmc_ar_logpsi",
            "vmc_ar_sample", "vmc_ar_local_energy", "vmc_ar_grad", "vmc_ar_sr_step",
            "vmc_cnn_set_params", "vmc_cnn_get_params", "vmc_cnn_eval", "vmc_cnn_grad",
            "vmc_cnn_sample", "vmc_cnn_sr_step"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libvmc.so and declare the signatures (raises OSError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libvmc.so not found at {path}; build it with "
                      "`python -m paper_2108_03409_b300.build`")
    lib = ctypes.CDLL(path)
    P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "vmc_init": (i32, [ctypes.POINTER(vmc_config), ctypes.POINTER(vmc_lattice), i32, P,
                           ctypes.POINTER(P)]),
        "vmc_destroy": (None, [P]),
        "vmc_last_error": (ctypes.c_char_p, [P]),
        "vmc_set_params": (i32, [P, i32, P]),
        "vmc_get_params": (i32, [P, i32, P]),
        "vmc_set_chains": (i32, [P, i32, P]),
        "vmc_get_chains": (i32, [P, i32, P]),
        "vmc_theta": (i32, [P, i32, P, i64, P]),
        "vmc_logpsi": (i32, [P, i32, P, i64, P]),
        "vmc_local_energy": (i32, [P, i32, P, i64, P]),
        "vmc_sample": (i32, [P, i32, i32, i32, P, P, P]),
        "vmc_grad": (i32, [P, i32, P, P, i64, P, P, P]),
        "vmc_qfm": (i32, [P, i32, P, i64, i32, P]),
        "vmc_solve": (i32, [P, i32, P, P, P, ctypes.POINTER(i32), ctypes.POINTER(f64)]),
        "vmc_sr_step": (i32, [P, i32, f64, ctypes.POINTER(vmc_sr_stats)]),
        "vmc_sr_step_on": (i32, [P, i32, P, i64, f64, ctypes.POINTER(vmc_sr_stats)]),
        "vmc_kernel_launches": (i64, [P]),
        "vmc_num_samples": (i64, [P]),
        "vmc_num_params": (i64, [P, i32]),
        "vmc_force_noalloc": (i32, [P, P, P, i64, i32, i32, P, P, P]),
        "vmc_cg_solve": (i32, [P, i32, P, i64, P, P, ctypes.POINTER(i32), ctypes.POINTER(f64)]),
        "vmc_sr_apply": (i32, [P, i32, P, i64, P, P]),
        "vmc_made_set_params": (i32, [P, i32, P]),
        "vmc_made_get_params": (i32, [P, i32, P]),
        "vmc_made_logq": (i32, [P, i32, P, i64, P]),
        "vmc_made_grad": (i32, [P, i32, P, i64, P, ctypes.POINTER(f64)]),
        "vmc_proposal_train": (i32, [P, i32, P, i64, i32, f64, ctypes.POINTER(f64)]),
        "vmc_made_sample": (i32, [P, i32, i64, ctypes.c_uint64, P, P]),
        "vmc_sample_learned": (i32, [P, i32, i32, P, P, ctypes.POINTER(f64)]),
        "vmc_sample_all": (i32, [P, i32, i32, P, P, i32, ctypes.POINTER(f64)]),
        "vmc_autotuned_warps_per_block": (i32, [P]),
        "vmc_autotuned_slots_per_lane": (i32, [P]),
        "vmc_get_state": (i32, [P, P, ctypes.POINTER(ctypes.c_size_t)]),
        "vmc_set_state": (i32, [P, P, ctypes.c_size_t]),
        "vmc_selftest_wait_timeout": (i32, [P, i32]),
        "vmc_tdvp_rhs": (i32, [P, i32, P, i64, P, ctypes.POINTER(vmc_tdvp_opts), P,
                               ctypes.POINTER(vmc_tdvp_stats)]),
        "vmc_tdvp_step": (i32, [P, i32, ctypes.POINTER(vmc_tdvp_opts), ctypes.POINTER(f64),
                                ctypes.POINTER(f64), ctypes.POINTER(vmc_tdvp_stats)]),
        "vmc_excited_lambda": (i32, [P, i32, i32, P, i64, i32, P]),
        "vmc_excited_rhs": (i32, [P, i32, i32, P, i64, P, ctypes.POINTER(vmc_tdvp_opts), P,
                                  ctypes.POINTER(vmc_excited_stats)]),
        "vmc_excited_step": (i32, [P, i32, i32, f64, ctypes.POINTER(vmc_tdvp_opts),
                                   ctypes.POINTER(vmc_excited_stats)]),
        "vmc_ar_set_params": (i32, [P, i32, P]),
        "vmc_ar_get_params": (i32, [P, i32, P]),
        "vmc_ar_logpsi": (i32, [P, i32, P, i64, P]),
        "vmc_ar_sample": (i32, [P, i32, i64, P, P]),
        "vmc_ar_local_energy": (i32, [P, i32, P, i64, P]),
        "vmc_ar_grad": (i32, [P, i32, P, P, i64, P, P, P, P]),
        "vmc_ar_sr_step": (i32, [P, i32, f64, ctypes.POINTER(vmc_sr_stats)]),
        "vmc_cnn_set_params": (i32, [P, i32, P]),
        "vmc_cnn_get_params": (i32, [P, i32, P]),
        "vmc_cnn_eval": (i32, [P, i32, P, i64, P, P]),
        "vmc_cnn_grad": (i32, [P, i32, P, i64, P]),
        "vmc_cnn_sample": (i32, [P, i32, i32, i32, P, P, P]),
        "vmc_cnn_sr_step": (i32, [P, i32, f64, ctypes.POINTER(vmc_tdvp_opts),
                                  ctypes.POINTER(vmc_tdvp_stats)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t) -> Optional[int]:
    """Raw device/host pointer of a torch tensor (or numpy array, or None)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        assert t.is_contiguous(), "tensors passed to libvmc must be contiguous"
        return t.data_ptr()
    return t.ctypes.data


def _check(ctx, status: int):
    if status != VMC_OK:
        msg = load().vmc_last_error(ctx).decode() if ctx else ""
        raise VmcError(status, msg)


def make_config(seed=1, n_chains=256, sweep_len=0, therm_sweeps=20, sweeps_per_sample=1,
                samples_per_chain=1, precision=PREC_FP32, solver=SOLVER_CHOLESKY_FP64,
                shift=1e-4, shift_mode=SHIFT_MULTIPLICATIVE, cg_maxit=100,
                cg_tol=1e-10, made_hidden=0, made_batch=0, tdvp=0, ar_ansatz=0,
                cnn_ansatz=0) -> vmc_config:
    return vmc_config(seed, n_chains, sweep_len, therm_sweeps, sweeps_per_sample,
                      samples_per_chain, precision, solver, shift, shift_mode, cg_maxit, cg_tol,
                      made_hidden, made_batch, tdvp, ar_ansatz, cnn_ansatz)


def make_tdvp_opts(gamma=1j, eps_pinv=0.0, pinv_soft=1, eps_snr=0.0, shift=0.0, exact=0,
                   eps_step=1e-6, tau_max=0.0, max_retries=0, jacobi_max_sweeps=0) -> vmc_tdvp_opts:
    g = complex(gamma)
    return vmc_tdvp_opts(g.real, g.imag, eps_pinv, pinv_soft, eps_snr, shift, exact, eps_step,
                         tau_max, max_retries, jacobi_max_sweeps)


def make_lattice(model, Lx, Ly=1, J=1.0, h=0.0, alpha=1) -> vmc_lattice:
    return vmc_lattice(model, Lx, Ly, J, h, alpha)


# --------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# --------------------------------------------------------------------------------------
def vmc_init(cfg: vmc_config, lattices: Sequence[vmc_lattice], stream: int = 0):
    lib = load()
    arr = (vmc_lattice * len(lattices))(*lattices)
    out = ctypes.c_void_p()
    st = lib.vmc_init(ctypes.byref(cfg), arr, len(lattices), ctypes.c_void_p(stream or None),
                      ctypes.byref(out))
    if st != VMC_OK:
        raise VmcError(st, "vmc_init failed")
    return out


def vmc_destroy(ctx):
    if ctx:
        load().vmc_destroy(ctx)


def vmc_set_params(ctx, lattice, params_host):
    """params_host: numpy complex128 [P]."""
    import numpy as np
    p = np.ascontiguousarray(params_host, dtype=np.complex128)
    _check(ctx, load().vmc_set_params(ctx, lattice, p.ctypes.data))


def vmc_get_params(ctx, lattice):
    import numpy as np
    P = load().vmc_num_params(ctx, lattice)
    out = np.zeros(P, dtype=np.complex128)
    _check(ctx, load().vmc_get_params(ctx, lattice, out.ctypes.data))
    return out


def vmc_set_chains(ctx, lattice, spins_host):
    import numpy as np
    s = np.ascontiguousarray(spins_host, dtype=np.int8)
    _check(ctx, load().vmc_set_chains(ctx, lattice, s.ctypes.data))


def vmc_get_chains(ctx, lattice, n_chains, N):
    import numpy as np
    out = np.zeros((n_chains, N), dtype=np.int8)
    _check(ctx, load().vmc_get_chains(ctx, lattice, out.ctypes.data))
    return out


def vmc_theta(ctx, lattice, spins, out):
    _check(ctx, load().vmc_theta(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(out)))


def vmc_logpsi(ctx, lattice, spins, out):
    _check(ctx, load().vmc_logpsi(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(out)))


def vmc_local_energy(ctx, lattice, spins, out):
    _check(ctx, load().vmc_local_energy(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(out)))


def vmc_sample(ctx, lattice, n_therm, n_samples, spins_out=None, logpsi_out=None, eloc_out=None):
    _check(ctx, load().vmc_sample(ctx, lattice, n_therm, n_samples, _ptr(spins_out),
                                  _ptr(logpsi_out), _ptr(eloc_out)))


def vmc_grad(ctx, lattice, spins, eloc, O_out=None, F_out=None, want_stats=True):
    import numpy as np
    es = np.zeros(4, dtype=np.float64) if want_stats else None
    _check(ctx, load().vmc_grad(ctx, lattice, _ptr(spins), _ptr(eloc), spins.shape[0],
                                _ptr(O_out), _ptr(F_out), None if es is None else es.ctypes.data))
    return es


def vmc_qfm(ctx, lattice, spins, precision, S_out):
    _check(ctx, load().vmc_qfm(ctx, lattice, _ptr(spins), spins.shape[0], precision, _ptr(S_out)))


def vmc_solve(ctx, lattice, S, F, x):
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    _check(ctx, load().vmc_solve(ctx, lattice, _ptr(S), _ptr(F), _ptr(x), ctypes.byref(it),
                                 ctypes.byref(rr)))
    return it.value, rr.value


def vmc_cg_solve(ctx, lattice, spins, F, x):
    """Matrix-free CG; raises VmcError (with ``iters`` and ``relres`` attributes) if cg_tol
    was not reached within cg_maxit iterations."""
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    try:
        _check(ctx, load().vmc_cg_solve(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(F),
                                        _ptr(x), ctypes.byref(it), ctypes.byref(rr)))
    except VmcError as e:
        e.iters, e.relres = it.value, rr.value
        raise
    return it.value, rr.value


def vmc_sr_apply(ctx, lattice, spins, v, y):
    """y = S~ v (the CG operator) for the sample set spins (dev int8 [n][N])."""
    _check(ctx, load().vmc_sr_apply(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(v), _ptr(y)))


def vmc_sr_step(ctx, lattice, dt) -> vmc_sr_stats:
    """One SR step.  A failed step raises VmcError; its ``stats`` attribute holds the step's
    statistics (e.g. solver_converged = 0 when the CG did not reach cg_tol)."""
    st = vmc_sr_stats()
    try:
        _check(ctx, load().vmc_sr_step(ctx, lattice, float(dt), ctypes.byref(st)))
    except VmcError as e:
        e.stats = st
        raise
    return st


def vmc_sr_step_on(ctx, lattice, spins, dt) -> vmc_sr_stats:
    """The SR step on a given sample set (dev int8 [n_chains * samples_per_chain][N])."""
    st = vmc_sr_stats()
    try:
        _check(ctx, load().vmc_sr_step_on(ctx, lattice, _ptr(spins), spins.shape[0], float(dt),
                                          ctypes.byref(st)))
    except VmcError as e:
        e.stats = st
        raise
    return st


def vmc_kernel_launches(ctx) -> int:
    return int(load().vmc_kernel_launches(ctx))


def vmc_num_samples(ctx) -> int:
    return int(load().vmc_num_samples(ctx))


def vmc_num_params(ctx, lattice) -> int:
    return int(load().vmc_num_params(ctx, lattice))


def vmc_force_noalloc(spins, tanh_theta, eloc, N, M, F_out, meanO_out=None, stream=0):
    """F (and optionally <O>) without device allocation; scratch is a fixed static array."""
    st = load().vmc_force_noalloc(_ptr(spins), _ptr(tanh_theta), _ptr(eloc), spins.shape[0], N, M,
                                  _ptr(F_out), _ptr(meanO_out), ctypes.c_void_p(stream or None))
    if st != VMC_OK:
        raise VmcError(st, "vmc_force_noalloc failed")


# --------------------------------------------------------------------------------------
# learned proposal
# --------------------------------------------------------------------------------------
def vmc_made_set_params(ctx, lattice, params_host):
    import numpy as np
    p = np.ascontiguousarray(params_host, dtype=np.float32)
    _check(ctx, load().vmc_made_set_params(ctx, lattice, p.ctypes.data))


def vmc_made_get_params(ctx, lattice, n_params):
    import numpy as np
    out = np.zeros(n_params, dtype=np.float32)
    _check(ctx, load().vmc_made_get_params(ctx, lattice, out.ctypes.data))
    return out


def vmc_made_logq(ctx, lattice, spins, out):
    _check(ctx, load().vmc_made_logq(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(out)))


def vmc_made_grad(ctx, lattice, spins, grad_out):
    loss = ctypes.c_double(0.0)
    _check(ctx, load().vmc_made_grad(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(grad_out),
                                     ctypes.byref(loss)))
    return loss.value


def vmc_proposal_train(ctx, lattice, samples, epochs, lr=1e-3):
    loss = ctypes.c_double(0.0)
    _check(ctx, load().vmc_proposal_train(ctx, lattice, _ptr(samples), samples.shape[0],
                                          int(epochs), float(lr), ctypes.byref(loss)))
    return loss.value


def vmc_made_sample(ctx, lattice, n, round_, spins_out, logq_out=None):
    _check(ctx, load().vmc_made_sample(ctx, lattice, int(n), int(round_), _ptr(spins_out),
                                       _ptr(logq_out)))


def vmc_sample_learned(ctx, lattice, n_rounds, spins_out=None, eloc_out=None):
    acc = ctypes.c_double(0.0)
    _check(ctx, load().vmc_sample_learned(ctx, lattice, int(n_rounds), _ptr(spins_out),
                                          _ptr(eloc_out), ctypes.byref(acc)))
    return acc.value


def vmc_sample_all(ctx, n_therm, n_samples, spins_out=None, eloc_out=None, use_graph=True):
    ms = ctypes.c_double(0.0)
    _check(ctx, load().vmc_sample_all(ctx, int(n_therm), int(n_samples), _ptr(spins_out),
                                      _ptr(eloc_out), 1 if use_graph else 0, ctypes.byref(ms)))
    return ms.value


def vmc_autotuned_warps_per_block(ctx) -> int:
    return int(load().vmc_autotuned_warps_per_block(ctx))


def vmc_autotuned_slots_per_lane(ctx) -> int:
    return int(load().vmc_autotuned_slots_per_lane(ctx))


def vmc_get_state(ctx) -> bytes:
    """Checkpoint of the context (parameters, chains, RNG counters, learned proposal)."""
    n = ctypes.c_size_t(0)
    _check(ctx, load().vmc_get_state(ctx, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, load().vmc_get_state(ctx, buf, ctypes.byref(n)))
    return buf.raw[:n.value]


def vmc_set_state(ctx, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(ctx, load().vmc_set_state(ctx, buf, len(state)))


def vmc_selftest_wait_timeout(ctx, which: int) -> int:
    """Run a bounded wait that nothing satisfies; returns the status (VMC_ERR_TIMEOUT expected)."""
    return int(load().vmc_selftest_wait_timeout(ctx, int(which)))


def vmc_tdvp_rhs(ctx, lattice, opts, thetadot, spins=None, weights=None) -> vmc_tdvp_stats:
    """thetadot (dev float64 [P][2]) of the current parameters; spins (dev int8 [n][N]) with
    optional weights (dev float64 [n]), or None: the context's own sample set."""
    st = vmc_tdvp_stats()
    n = spins.shape[0] if spins is not None else 0
    _check(ctx, load().vmc_tdvp_rhs(ctx, lattice, _ptr(spins), n, _ptr(weights),
                                    ctypes.byref(opts), _ptr(thetadot), ctypes.byref(st)))
    return st


def vmc_tdvp_step(ctx, lattice, opts, t, tau):
    """One accepted adaptive Heun step; returns (t, tau_next, stats)."""
    tt, hh = ctypes.c_double(t), ctypes.c_double(tau)
    st = vmc_tdvp_stats()
    _check(ctx, load().vmc_tdvp_step(ctx, lattice, ctypes.byref(opts), ctypes.byref(tt),
                                     ctypes.byref(hh), ctypes.byref(st)))
    return tt.value, hh.value, st


def vmc_excited_lambda(ctx, lattice, ref_lattice, spins_phi=None, exact=0) -> complex:
    """lambda = <psi/phi> over |phi|^2 (caller's samples, Metropolis samples or exact sums)."""
    import numpy as np
    out = np.zeros(2, dtype=np.float64)
    n = spins_phi.shape[0] if spins_phi is not None else 0
    _check(ctx, load().vmc_excited_lambda(ctx, lattice, ref_lattice, _ptr(spins_phi), n, int(exact),
                                          out.ctypes.data))
    return complex(out[0], out[1])


def vmc_excited_rhs(ctx, lattice, ref_lattice, opts, thetadot, spins_psi=None, lam=None):
    import numpy as np
    st = vmc_excited_stats()
    n = spins_psi.shape[0] if spins_psi is not None else 0
    la = None if lam is None else np.array([complex(lam).real, complex(lam).imag], np.float64)
    _check(ctx, load().vmc_excited_rhs(ctx, lattice, ref_lattice, _ptr(spins_psi), n,
                                       None if la is None else la.ctypes.data, ctypes.byref(opts),
                                       _ptr(thetadot), ctypes.byref(st)))
    return st


def vmc_excited_step(ctx, lattice, ref_lattice, dt, opts) -> vmc_excited_stats:
    st = vmc_excited_stats()
    _check(ctx, load().vmc_excited_step(ctx, lattice, ref_lattice, float(dt), ctypes.byref(opts),
                                        ctypes.byref(st)))
    return st


# ---- the autoregressive network as the ansatz -------------------------------------------
def vmc_ar_set_params(ctx, lattice, params_host):
    """params_host: numpy float64 [P] (canonical layout of the masked network)."""
    import numpy as np
    p = np.ascontiguousarray(params_host, dtype=np.float64)
    _check(ctx, load().vmc_ar_set_params(ctx, lattice, p.ctypes.data))


def vmc_ar_get_params(ctx, lattice, P):
    import numpy as np
    out = np.zeros(P, dtype=np.float64)
    _check(ctx, load().vmc_ar_get_params(ctx, lattice, out.ctypes.data))
    return out


def vmc_ar_logpsi(ctx, lattice, spins, logpsi):
    _check(ctx, load().vmc_ar_logpsi(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(logpsi)))


def vmc_ar_sample(ctx, lattice, spins_out, logpsi_out=None):
    _check(ctx, load().vmc_ar_sample(ctx, lattice, spins_out.shape[0], _ptr(spins_out),
                                     _ptr(logpsi_out)))


def vmc_ar_local_energy(ctx, lattice, spins, eloc):
    _check(ctx, load().vmc_ar_local_energy(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(eloc)))


def vmc_ar_grad(ctx, lattice, spins, eloc, O_out=None, meanO_out=None, F_out=None):
    import numpy as np
    es = np.zeros(4, dtype=np.float64)
    _check(ctx, load().vmc_ar_grad(ctx, lattice, _ptr(spins), _ptr(eloc), spins.shape[0],
                                   _ptr(O_out), _ptr(meanO_out), _ptr(F_out), es.ctypes.data))
    return es


def vmc_ar_sr_step(ctx, lattice, dt) -> vmc_sr_stats:
    st = vmc_sr_stats()
    _check(ctx, load().vmc_ar_sr_step(ctx, lattice, float(dt), ctypes.byref(st)))
    return st


# ---- the translation-symmetric CNN-ELU ansatz --------------------------------------------
def vmc_cnn_set_params(ctx, lattice, params_host):
    import numpy as np
    p = np.ascontiguousarray(params_host, dtype=np.float64)
    _check(ctx, load().vmc_cnn_set_params(ctx, lattice, p.ctypes.data))


def vmc_cnn_get_params(ctx, lattice, P):
    import numpy as np
    out = np.zeros(P, dtype=np.float64)
    _check(ctx, load().vmc_cnn_get_params(ctx, lattice, out.ctypes.data))
    return out


def vmc_cnn_eval(ctx, lattice, spins, logpsi=None, eloc=None):
    _check(ctx, load().vmc_cnn_eval(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(logpsi),
                                    _ptr(eloc)))


def vmc_cnn_grad(ctx, lattice, spins, O_out):
    _check(ctx, load().vmc_cnn_grad(ctx, lattice, _ptr(spins), spins.shape[0], _ptr(O_out)))


def vmc_cnn_sample(ctx, lattice, n_therm, n_samples, spins_out=None, logpsi_out=None,
                   eloc_out=None):
    _check(ctx, load().vmc_cnn_sample(ctx, lattice, n_therm, n_samples, _ptr(spins_out),
                                      _ptr(logpsi_out), _ptr(eloc_out)))


def vmc_cnn_sr_step(ctx, lattice, dt, opts) -> vmc_tdvp_stats:
    st = vmc_tdvp_stats()
    _check(ctx, load().vmc_cnn_sr_step(ctx, lattice, float(dt), ctypes.byref(opts), ctypes.byref(st)))
    return st
