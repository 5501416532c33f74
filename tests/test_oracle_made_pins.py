"""Pins of the oracle's MADE proposal (masked autoregressive MLP, Germain et al. 2015)
against what the definition fixes: the autoregressive property, normalisation, the
conditionals, finite-difference gradients, Adam's closed forms and exact sampling."""
import numpy as np
import pytest

import oracle
from paper_2108_03409_b300 import inputs


def _params(N, H, scale, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, oracle.made_nparams(N, H))


def test_made_is_autoregressive():
    """z_d depends on s_1 .. s_{d-1} only: flipping any later site leaves it bit-identical."""
    N, H = 9, 20
    p = _params(N, H, 0.7, 1)
    s = inputs.random_spins(16, N, seed=2)
    _, z = oracle.made_forward(N, H, p, s, want_z=True)
    for j in range(N):
        t = s.copy()
        t[:, j] *= -1
        _, zt = oracle.made_forward(N, H, p, t, want_z=True)
        assert np.array_equal(z[:, :j + 1], zt[:, :j + 1])      # z_1 .. z_{j+1} (1-based)


def test_made_normalised_and_conditionals_by_enumeration():
    """sum_s q(s) = 1, and sigma(z_d) equals the conditional of q computed by brute-force
    marginalisation over the later sites."""
    N, H = 8, 16
    p = _params(N, H, 0.8, 3)
    S = oracle.all_states(N)
    lq, z = oracle.made_forward(N, H, p, S, want_z=True)
    q = np.exp(lq)
    assert abs(q.sum() - 1.0) <= 1e-12
    bits = (1 - S) // 2
    for k in range(0, len(S), 37):
        s = S[k]
        for d in range(N):
            prefix = np.all(S[:, :d] == s[:d], axis=1)
            den = q[prefix].sum()
            num = q[prefix & (S[:, d] == 1)].sum()
            assert abs(num / den - 1.0 / (1.0 + np.exp(-z[k, d]))) <= 1e-12


def test_made_grad_central_differences():
    N, H = 6, 10
    p = _params(N, H, 0.5, 4)
    s = inputs.random_spins(40, N, seed=5)
    g, L = oracle.made_grad(N, H, p, s)
    assert abs(L + oracle.made_forward(N, H, p, s).mean()) <= 1e-12
    eps = 1e-6
    for k in range(p.size):
        pp = p.copy(); pp[k] += eps
        pm = p.copy(); pm[k] -= eps
        fd = (-oracle.made_forward(N, H, pp, s).mean() + oracle.made_forward(N, H, pm, s).mean()) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-8 * max(1.0, abs(g[k]))
    # masked-out weights have exactly zero gradient
    W1 = g[:H * N].reshape(H, N)
    deg = np.arange(H) % (N - 1) + 1
    for kk in range(H):
        assert np.all(W1[kk, deg[kk]:] == 0.0)


def test_adam_closed_forms():
    """With a constant gradient the bias-corrected moments are exact, so every step moves
    theta by -lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    t0 = th.copy()
    for t in range(1, 6):
        th, m, v = oracle.adam_step(th, m, v, g, t, lr=1e-2)
        assert np.allclose(th, t0 - t * 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2])
def test_made_sampler_chi2(seed):
    """Exact autoregressive sampling: the histogram of 16384 draws matches q at N = 10."""
    from scipy.stats import chi2
    N, H = 10, 16
    p = _params(N, H, 0.6, 10 + seed)
    n = 16384
    s, lq, _ = oracle.made_sample(N, H, p, n, seed=seed)
    assert np.allclose(lq, oracle.made_forward(N, H, p, s), atol=1e-12)
    S = oracle.all_states(N)
    q = np.exp(oracle.made_forward(N, H, p, S))
    idx = (((1 - s.astype(np.int64)) // 2) << np.arange(N)).sum(axis=1)
    counts = np.bincount(idx, minlength=1 << N)
    exp = q * n
    order = np.argsort(exp)
    c_m, e_m, ac, ae = [], [], 0.0, 0.0
    for k in order:
        ac += counts[k]; ae += exp[k]
        if ae >= 5:
            c_m.append(ac); e_m.append(ae); ac = ae = 0.0
    c_m[-1] += ac; e_m[-1] += ae
    c_m, e_m = np.array(c_m), np.array(e_m)
    assert chi2.sf(np.sum((c_m - e_m) ** 2 / e_m), len(c_m) - 1) > 1e-3
