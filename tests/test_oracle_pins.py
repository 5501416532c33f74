"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests retypes the oracle's formulas: each compares it with an independent
route to the same number (brute force over hidden units, a dense Hamiltonian built from
bit operations, finite differences, a library routine, a closed form or an invariant).
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_2108_03409_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------------------
# independent Hamiltonian construction (bit operations on basis indices; bit 0 <-> s=+1)
# --------------------------------------------------------------------------------------
def _neighbours(Lx, Ly):
    out = []
    for y in range(Ly):
        for x in range(Lx):
            out.append((x + Lx * y, (x + 1) % Lx + Lx * y))
    if Ly > 1:
        for y in range(Ly):
            for x in range(Lx):
                out.append((x + Lx * y, x + Lx * ((y + 1) % Ly)))
    return out


def _dense_h(model, Lx, Ly, J, h):
    N = Lx * Ly
    D = 1 << N
    idx = np.arange(D, dtype=np.int64)
    spin = 1 - 2 * ((idx[:, None] >> np.arange(N)[None, :]) & 1)
    rows, cols, vals = [], [], []
    diag = np.zeros(D)
    for (i, j) in _neighbours(Lx, Ly):
        zz = spin[:, i] * spin[:, j]
        if model == inputs.MODEL_TFIM:
            diag += -J * zz
        else:
            diag += J * zz
            anti = zz < 0
            src = idx[anti]
            dst = src ^ ((1 << i) | (1 << j))
            rows.append(dst); cols.append(src); vals.append(np.full(src.size, 2.0 * J))
    if model == inputs.MODEL_TFIM:
        for i in range(N):
            rows.append(idx ^ (1 << i)); cols.append(idx); vals.append(np.full(D, -h))
    rows.append(idx); cols.append(idx); vals.append(diag)
    H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(D, D))
    return H


def _state_index(s):
    bits = (1 - s.astype(np.int64)) // 2
    return (bits << np.arange(s.shape[1])[None, :]).sum(axis=1)


# --------------------------------------------------------------------------------------
# RNG
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((123, 456), (7, 0, 3, 0)),
                                     ((2**64 - 1, 17), (5, 2**63, 11, 9))])
def test_philox4x64_matches_numpy(key, ctr):
    """numpy.random.Philox is Philox4x64-10; it increments the counter before each block."""
    pre = np.array(ctr, dtype=np.uint64)
    # numpy adds one to the 256-bit counter before producing a block
    carry = np.zeros(4, dtype=np.uint64)
    val = int(ctr[0]) + (int(ctr[1]) << 64) + (int(ctr[2]) << 128) + (int(ctr[3]) << 192)
    val = (val - 1) % (1 << 256)
    for w in range(4):
        carry[w] = (val >> (64 * w)) & (2**64 - 1)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=carry)
    ref = bg.random_raw(4)
    got = oracle.philox4x64(pre, key)
    assert np.array_equal(ref.astype(np.uint64), got)


# --------------------------------------------------------------------------------------
# log psi
# --------------------------------------------------------------------------------------
def test_logpsi_equals_sum_over_hidden_units():
    """The RBM amplitude is the marginal of exp(a.s + b.h + h.W.s) over hidden h = +-1:
    sum_h exp(...) = 2^M exp(log psi(s)).  Brute force over all 2^M hidden states."""
    N, M = 4, 5
    p = inputs.rbm_params(N, M, 0.4, seed=5)
    a, b, W = p[:N], p[N:N + M], p[N + M:].reshape(M, N)
    S = oracle.all_states(N)
    H = oracle.all_states(M)
    lp = oracle.logpsi(N, M, p, S)
    for k, s in enumerate(S):
        e = np.exp(a @ s + H @ b + np.einsum("hj,ji,i->h", H, W, s))
        ref = e.sum()
        got = (2.0 ** M) * np.exp(lp[k])
        assert abs(got - ref) <= 1e-12 * abs(ref)


def test_theta_invariants_and_log_derivative():
    """theta of the oracle against what its definition fixes without retyping it: it is
    affine in s (theta(s) + theta(-s) = 2 b), a flip of site i changes theta_j by
    2 s_i W_ji with W read from the documented parameter layout [a | b | W (M x N)], and
    d log psi / d b_j = tanh theta_j by central finite differences of log psi."""
    N, M = 9, 6
    p = inputs.rbm_params(N, M, 0.4, seed=21)          # complex [a | b | W]
    b = p[N:N + M]
    W = p[N + M:].reshape(M, N)
    s = inputs.random_spins(7, N, seed=22)
    th = oracle.theta(N, M, p, s)
    assert np.allclose(th + oracle.theta(N, M, p, -s), 2 * b[None, :], atol=1e-13)
    for i in (0, 4, N - 1):
        sf = s.copy()
        sf[:, i] *= -1
        d = th - oracle.theta(N, M, p, sf)
        assert np.allclose(d, 2 * s[:, i, None] * W[None, :, i], atol=1e-13)
    eps = 1e-6
    for j in (0, M - 1):
        for unit in (1.0, 1j):
            dp = np.zeros_like(p)
            dp[N + j] = eps * unit
            fd = (oracle.logpsi(N, M, p + dp, s) - oracle.logpsi(N, M, p - dp, s)) / (2 * eps * unit)
            assert np.allclose(fd, np.tanh(th[:, j]), atol=1e-8)


@pytest.mark.parametrize("z", [0.3 + 0.2j, -45.0 + 3.0j, 400.0 - 7.5j, -2.0 + 1.5707j, 1e-9 + 0j])
def test_logcosh_against_high_precision(z):
    """N = 1, M = 1, a = 0, W = 0: log psi = log cosh(b).  Compared with mpmath at 50 digits,
    imaginary part mod 2 pi (the branch of the complex log is not fixed by psi)."""
    import mpmath
    mpmath.mp.dps = 50
    p = np.array([0.0, z, 0.0], dtype=np.complex128)
    got = oracle.logpsi(1, 1, p, np.array([[1]], np.int8))[0]
    ref = complex(mpmath.log(mpmath.cosh(mpmath.mpc(z.real, z.imag))))
    assert abs(got.real - ref.real) <= 1e-12 * max(1.0, abs(ref.real))
    dphi = (got.imag - ref.imag + math.pi) % (2 * math.pi) - math.pi
    assert abs(dphi) <= 1e-10


# --------------------------------------------------------------------------------------
# operator mapping and local energy
# --------------------------------------------------------------------------------------
def test_sx_worked_example():
    """The paper's sigma^x example (golden file), reproduced with the TFIM's X term:
    J = 0 removes the diagonal, h = -1 makes the X_1 element +1."""
    lines = [l.split() for l in open(os.path.join(HERE, "golden", "sx_example.txt"))
             if l.strip() and not l.startswith("#")]
    d = {l[0]: l[1:] for l in lines}
    site = int(d["site"][0])
    s_in = np.array([int(v) for v in d["input"]], np.int8)
    s_out = np.array([int(v) for v in d["output"]], np.int8)
    el = complex(float(d["element"][0]), float(d["element"][1]))
    sps, els = oracle.connected(inputs.MODEL_TFIM, 4, 1, 0.0, -1.0, s_in)
    assert els[0] == 0.0                                  # diagonal entry, J = 0
    hit = [k for k in range(1, len(sps)) if np.array_equal(sps[k], s_out)]
    assert len(hit) == 1
    assert els[hit[0]] == el
    assert np.sum(sps[hit[0]] != s_in) == 1 and sps[hit[0]][site] == -s_in[site]


@pytest.mark.parametrize("model,Lx,Ly,J,h,alpha,sigma", [
    (inputs.MODEL_TFIM, 8, 1, 1.0, 0.7, 1, 0.3),
    (inputs.MODEL_TFIM, 3, 3, 1.0, 2.5, 2, 0.2),
    (inputs.MODEL_HEIS, 10, 1, 1.0, 0.0, 1, 0.3),
    (inputs.MODEL_HEIS, 4, 4, 1.0, 0.0, 1, 0.1),
])
def test_eloc_equals_dense_hamiltonian_action(model, Lx, Ly, J, h, alpha, sigma):
    """E_loc(s) = (H psi)(s) / psi(s) for every enumerated s, with H built independently;
    and sum_s p(s) E_loc(s) = <psi|H|psi>/<psi|psi> (Eq. expectation_value)."""
    N = Lx * Ly
    M = alpha * N
    heis = model == inputs.MODEL_HEIS
    p = inputs.rbm_params(N, M, sigma, seed=11, marshall=(Lx, Ly) if heis else None)
    H = _dense_h(model, Lx, Ly, J, h)
    full = oracle.all_states(N)
    lp_full = oracle.logpsi(N, M, p, full)
    shift = lp_full.real.max()
    psi = np.exp(lp_full - shift)
    Hpsi = H @ psi
    S = oracle.all_states(N, sz0=heis)
    if S.shape[0] > 4000:
        S = S[np.random.default_rng(0).choice(S.shape[0], 4000, replace=False)]
    e = oracle.eloc(model, Lx, Ly, J, h, M, p, S)
    ix = _state_index(S)
    ref = Hpsi[ix] / psi[ix]
    assert np.max(np.abs(e - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))
    E, _, _, _ = oracle.exact_energy(model, Lx, Ly, J, h, M, p, sz0=heis)
    if heis:                       # H conserves Sz: restrict psi to the Sz = 0 sector
        psi = np.where(full.sum(axis=1) == 0, psi, 0.0)
        Hpsi = H @ psi
    Eref = np.vdot(psi, Hpsi) / np.vdot(psi, psi)
    assert abs(E - Eref) <= 1e-12 * abs(Eref)


def test_eloc_product_state_closed_form():
    """W = 0, b = 0: psi = prod_i exp(a_i s_i), so <Z_i> = tanh(2 Re a_i) and
    <X_i> = cos(2 Im a_i) / cosh(2 Re a_i);  E = -J sum <Z_i><Z_j> - h sum <X_i>."""
    Lx, Ly, J, h, M = 3, 3, 0.8, 1.7, 4
    N = Lx * Ly
    rng = np.random.default_rng(3)
    p = np.zeros(N + M + N * M, np.complex128)
    p[:N] = rng.normal(0, 0.4, N) + 1j * rng.normal(0, 0.9, N)
    E, _, _, _ = oracle.exact_energy(inputs.MODEL_TFIM, Lx, Ly, J, h, M, p)
    z = np.tanh(2 * p[:N].real)
    x = np.cos(2 * p[:N].imag) / np.cosh(2 * p[:N].real)
    ref = -J * sum(z[i] * z[j] for i, j in _neighbours(Lx, Ly)) - h * x.sum()
    assert abs(E - ref) <= 1e-12 * abs(ref)


def test_eloc_zero_variance_in_eigenstate():
    """J = 0 and psi = const is the eigenstate of -h sum X with energy -hN: the local energy
    is -hN on every configuration, so its variance vanishes."""
    N, M, h = 10, 10, 1.3
    p = np.zeros(N + M + N * M, np.complex128)
    S = oracle.all_states(N)
    e = oracle.eloc(inputs.MODEL_TFIM, N, 1, 0.0, h, M, p, S)
    assert np.max(np.abs(e - (-h * N))) <= 1e-12


# --------------------------------------------------------------------------------------
# log-derivatives
# --------------------------------------------------------------------------------------
def test_ok_central_finite_differences():
    """O_k = d log psi / d theta_k; holomorphy means real and imaginary steps agree."""
    N, M = 5, 6
    p = inputs.rbm_params(N, M, 0.3, seed=21)
    S = inputs.random_spins(7, N, seed=2)
    O = oracle.ok(N, M, p, S)
    eps = 1e-6
    for k in range(p.size):
        for step in (eps, 1j * eps):
            pp = p.copy(); pp[k] += step
            pm = p.copy(); pm[k] -= step
            fd = (oracle.logpsi(N, M, pp, S) - oracle.logpsi(N, M, pm, S)) / (2 * step)
            assert np.max(np.abs(fd - O[:, k])) <= 1e-8


# --------------------------------------------------------------------------------------
# S and F
# --------------------------------------------------------------------------------------
def test_sr_matrices_equal_numpy_covariance():
    """S_kl = <O_k^* O_l>^c and F_k = <O_k^* E>^c are population covariances; numpy.cov
    (bias=True) computes E[(x - x.mean) conj(y - y.mean)]."""
    rng = np.random.default_rng(4)
    Ns, P = 200, 9
    O = rng.normal(size=(Ns, P)) + 1j * rng.normal(size=(Ns, P))
    E = rng.normal(size=Ns) + 1j * rng.normal(size=Ns)
    S, F, Em = oracle.sr_matrices(O, E)
    C = np.cov(np.concatenate([O, E[:, None]], axis=1).T, bias=True)   # C[i,j]=E[x_i conj(x_j)]^c
    assert np.allclose(S, C[:P, :P].conj(), atol=1e-12)
    assert np.allclose(F, C[P, :P], atol=1e-12)
    assert abs(Em - E.mean()) < 1e-14
    s_e, f_e = oracle.sr_entries(O, E, [0, 3, 8], [5, 3, 1], [2, 7])
    assert np.allclose(s_e, S[[0, 3, 8], [5, 3, 1]], atol=1e-12)
    assert np.allclose(f_e, F[[2, 7]], atol=1e-12)


def test_force_is_half_the_exact_energy_gradient():
    """dE/dRe(theta_k) = 2 Re F_k and dE/dIm(theta_k) = 2 Im F_k (Eq. energy_gradient for a
    holomorphic ansatz), with E and F from exact enumeration."""
    Lx, Ly, J, h, M = 6, 1, 1.0, 0.9, 6
    N = Lx * Ly
    p = inputs.rbm_params(N, M, 0.25, seed=8)
    S, F, E = oracle.exact_sr(inputs.MODEL_TFIM, Lx, Ly, J, h, M, p)
    eps = 1e-5
    for k in range(p.size):
        for step, part in ((eps, F[k].real), (1j * eps, F[k].imag)):
            pp = p.copy(); pp[k] += step
            pm = p.copy(); pm[k] -= step
            Ep = oracle.exact_energy(inputs.MODEL_TFIM, Lx, Ly, J, h, M, pp)[0].real
            Emn = oracle.exact_energy(inputs.MODEL_TFIM, Lx, Ly, J, h, M, pm)[0].real
            assert abs((Ep - Emn) / (2 * eps) - 2 * part) <= 1e-7


def test_qfm_is_the_fubini_study_metric():
    """1 - |<psi|psi'>|^2 / (<psi|psi><psi'|psi'>) = eps^2 v^H S v + O(eps^3) for
    psi' = psi(theta + eps v) (Eq. qfm: S is the Fubini-Study metric tensor)."""
    Lx, Ly, J, h, M = 6, 1, 1.0, 0.9, 6
    N = Lx * Ly
    p = inputs.rbm_params(N, M, 0.25, seed=9)
    S, _, _ = oracle.exact_sr(inputs.MODEL_TFIM, Lx, Ly, J, h, M, p)
    full = oracle.all_states(N)
    rng = np.random.default_rng(1)
    for _ in range(3):
        v = rng.normal(size=p.size) + 1j * rng.normal(size=p.size)
        eps = 1e-4
        a = np.exp(oracle.logpsi(N, M, p, full))
        b = np.exp(oracle.logpsi(N, M, p + eps * v, full))
        inf = 1 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)
        pred = eps ** 2 * np.vdot(v, S @ v).real
        assert abs(inf - pred) <= 1e-3 * pred


def test_qfm_hermitian_psd_and_sz0_null_mode():
    """S is Hermitian PSD; in the Sz = 0 sector sum_i O_{a_i} = sum_i s_i = 0, so the vector
    with ones on the a-block is an exact null vector of S."""
    Lx, Ly, alpha = 4, 4, 1
    N, M = Lx * Ly, alpha * Lx * Ly
    p = inputs.rbm_params(N, M, 0.1, seed=3, marshall=(Lx, Ly))
    S = inputs.random_sz0_spins(300, N, seed=4)
    O = oracle.ok(N, M, p, S)
    E = oracle.eloc(inputs.MODEL_HEIS, Lx, Ly, 1.0, 0.0, M, p, S)
    Sm, F, _ = oracle.sr_matrices(O, E)
    assert np.allclose(Sm, Sm.conj().T, atol=1e-13)
    assert np.linalg.eigvalsh(Sm).min() > -1e-10
    v = np.zeros(Sm.shape[0], np.complex128)
    v[:N] = 1.0
    assert np.linalg.norm(Sm @ v) <= 1e-12


# --------------------------------------------------------------------------------------
# shift and solves
# --------------------------------------------------------------------------------------
def test_shift_modes():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
    S = A @ A.conj().T
    m = oracle.shift(S, 0.1, 0)
    a = oracle.shift(S, 0.1, 1)
    assert np.allclose(np.diag(m), 1.1 * np.diag(S), rtol=0, atol=1e-14)
    assert np.allclose(np.diag(a), np.diag(S) + 0.1, rtol=0, atol=1e-14)
    off = ~np.eye(5, dtype=bool)
    assert np.array_equal(m[off], S[off]) and np.array_equal(a[off], S[off])


def test_cholesky_solve_against_numpy():
    rng = np.random.default_rng(7)
    n = 60
    A = rng.normal(size=(n, 40)) + 1j * rng.normal(size=(n, 40))
    S = oracle.shift(A @ A.conj().T / 40, 1e-3, 0)
    F = rng.normal(size=n) + 1j * rng.normal(size=n)
    x = oracle.cholesky_solve(S, F)
    assert np.linalg.norm(S @ x - F) <= 1e-12 * np.linalg.norm(F) * np.linalg.cond(S)
    assert np.allclose(x, np.linalg.solve(S, F), rtol=1e-9, atol=0)


def test_cholesky_rejects_indefinite():
    S = np.diag([1.0, -1.0, 2.0]).astype(np.complex128)
    with pytest.raises(oracle.OracleError):
        oracle.cholesky_solve(S, np.ones(3, np.complex128))


@pytest.mark.parametrize("mode", [0, 1])
def test_sr_apply_matches_dense_shifted_s(mode):
    """The matrix-free operator equals the dense shifted S (formed by the separately pinned
    sr_matrices) times v, and v^H S~ v is real and positive."""
    rng = np.random.default_rng(17)
    Ns, P = 60, 25
    O = rng.normal(size=(Ns, P)) + 1j * rng.normal(size=(Ns, P)) + 0.7   # non-zero mean
    v = rng.normal(size=P) + 1j * rng.normal(size=P)
    S, _, _ = oracle.sr_matrices(O, np.zeros(Ns))
    y = oracle.sr_apply(O, v, 1e-2, mode)
    yd = oracle.shift(S, 1e-2, mode) @ v
    assert np.linalg.norm(y - yd) <= 1e-12 * np.linalg.norm(yd)
    q = np.vdot(v, y)
    assert q.real > 0 and abs(q.imag) <= 1e-12 * abs(q)


@pytest.mark.parametrize("mode", [0, 1])
def test_cg_matches_dense_solve(mode):
    rng = np.random.default_rng(5)
    Ns, P = 50, 30
    O = rng.normal(size=(Ns, P)) + 1j * rng.normal(size=(Ns, P))
    E = rng.normal(size=Ns) + 1j * rng.normal(size=Ns)
    S, F, _ = oracle.sr_matrices(O, E)
    St = oracle.shift(S, 1e-2, mode)
    xd = np.linalg.solve(St, F)
    x, it, rr = oracle.cg_solve(O, F, 1e-2, mode, tol=1e-12, maxit=500)
    assert rr <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


# --------------------------------------------------------------------------------------
# Metropolis: the stationary distribution is |psi|^2
# --------------------------------------------------------------------------------------
def _chi2_pvalue(counts, probs, n):
    from scipy.stats import chi2
    exp = probs * n
    order = np.argsort(exp)
    # merge the smallest-expectation bins until every merged bin expects >= 5 counts
    c_m, e_m = [], []
    acc_c = acc_e = 0.0
    for k in order:
        acc_c += counts[k]; acc_e += exp[k]
        if acc_e >= 5.0:
            c_m.append(acc_c); e_m.append(acc_e); acc_c = acc_e = 0.0
    if acc_e > 0:
        c_m[-1] += acc_c; e_m[-1] += acc_e
    c_m, e_m = np.array(c_m), np.array(e_m)
    stat = np.sum((c_m - e_m) ** 2 / e_m)
    return chi2.sf(stat, len(c_m) - 1)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_metropolis_tfim_histogram_chi2(seed):
    """Independent chains (final state after 40 sweeps from random starts) are iid draws
    from |psi|^2: chi-square against exact enumeration at N = 10."""
    N, M = 10, 10
    p = inputs.rbm_params(N, M, 0.2, seed=100 + seed)
    C = 16384
    s0 = inputs.random_spins(C, N, seed=seed)
    s, _, _, acc = oracle.metropolis(inputs.MODEL_TFIM, N, 1, M, p, s0, seed=seed, n_sweeps=40)
    full = oracle.all_states(N)
    prob = oracle.born_weights(oracle.logpsi(N, M, p, full))
    counts = np.bincount(_state_index(s), minlength=1 << N)
    assert _chi2_pvalue(counts, prob, C) > 1e-3


def test_metropolis_heisenberg_exchange_histogram_chi2():
    """Exchange moves keep Sz = 0 and sample |psi|^2 within the sector (chain N = 10)."""
    N, M = 10, 10
    p = inputs.rbm_params(N, M, 0.1, seed=77, marshall=(N, 1))
    C = 16384
    s0 = inputs.random_sz0_spins(C, N, seed=5)
    s, _, _, _ = oracle.metropolis(inputs.MODEL_HEIS, N, 1, M, p, s0, seed=9, n_sweeps=100)
    assert np.all(s.sum(axis=1) == 0)
    S = oracle.all_states(N, sz0=True)
    prob = oracle.born_weights(oracle.logpsi(N, M, p, S))
    lut = {int(k): n for n, k in enumerate(_state_index(S))}
    counts = np.bincount([lut[int(k)] for k in _state_index(s)], minlength=S.shape[0])
    assert _chi2_pvalue(counts, prob, C) > 1e-3


def test_metropolis_restart_is_seamless():
    """Counter-based RNG: 2k sweeps equal k sweeps, then k more sweeps from sweep0 = k."""
    N, M = 8, 8
    p = inputs.rbm_params(N, M, 0.3, seed=1)
    s0 = inputs.random_spins(32, N, seed=1)
    a, _, _, _ = oracle.metropolis(inputs.MODEL_TFIM, N, 1, M, p, s0, seed=4, n_sweeps=6)
    b, _, _, _ = oracle.metropolis(inputs.MODEL_TFIM, N, 1, M, p, s0, seed=4, n_sweeps=3)
    b, _, _, _ = oracle.metropolis(inputs.MODEL_TFIM, N, 1, M, p, b, seed=4, sweep0=3, n_sweeps=3)
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------------------
# tau_int
# --------------------------------------------------------------------------------------
def test_tau_int_ar1_closed_form():
    """AR(1) x_t = rho x_{t-1} + noise has rho(t) = rho^t, tau_int = (1+rho) / (2(1-rho))."""
    rng = np.random.default_rng(0)
    rho, n = 0.8, 400_000
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0]
    for t in range(1, n):
        x[t] = rho * x[t - 1] + e[t]
    ref = (1 + rho) / (2 * (1 - rho))
    assert abs(oracle.tau_int(x) - ref) <= 0.05 * ref


# --------------------------------------------------------------------------------------
# SR trajectory: imaginary-time TDVP reaches the Jordan-Wigner ground energy
# --------------------------------------------------------------------------------------
def jordan_wigner_e0(N, J, h):
    """Ground energy of the periodic TFIM chain -J sum ZZ - h sum X (even N): free fermions
    in the antiperiodic sector, E0 = -sum_n sqrt(J^2 + h^2 - 2 J h cos k_n), k_n = (2n+1) pi / N."""
    k = (2 * np.arange(N) + 1) * np.pi / N
    return -np.sum(np.sqrt(J * J + h * h - 2 * J * h * np.cos(k)))


@pytest.mark.parametrize("N,J,h", [(6, 1.0, 1.0), (8, 1.0, 0.7), (10, 1.0, 1.0)])
def test_jordan_wigner_matches_dense_ed(N, J, h):
    H = _dense_h(inputs.MODEL_TFIM, N, 1, J, h).toarray()
    e0 = np.linalg.eigvalsh(H)[0]
    assert abs(jordan_wigner_e0(N, J, h) - e0) <= 1e-10


def test_exact_sr_converges_to_jordan_wigner():
    """SR = imaginary-time TDVP Euler steps theta <- theta - dt S~^-1 F with exact S, F
    (no sampling noise) drives the alpha = 1 RBM of the N = 10 chain at J = h = 1 to within
    1e-3 of the Jordan-Wigner ground energy."""
    N, M, J, h = 10, 10, 1.0, 1.0
    E0 = jordan_wigner_e0(N, J, h)
    assert abs(E0 - (-12.784906443)) < 1e-8
    p = inputs.rbm_params(N, M, 0.01, seed=1234)
    E_prev = None
    for step in range(3000):
        S, F, E = oracle.exact_sr(inputs.MODEL_TFIM, N, 1, J, h, M, p)
        if abs(E.real - E0) / abs(E0) <= 1e-3:
            break
        x = oracle.cholesky_solve(oracle.shift(S, 1e-4, 0), F)
        p = oracle.update(p, x, 0.05)
        E_prev = E.real
    assert abs(E.real - E0) / abs(E0) <= 1e-3, (step, E.real, E0)
