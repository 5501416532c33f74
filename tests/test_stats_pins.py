"""Pins of the package's host-side statistics (paper_2108_03409_b300.stats), which the
benchmark uses for the effective-sample denominator 2 tau_int(E): against the oracle's
direct-sum Sokal estimator and against the AR(1) closed form."""
import numpy as np

import oracle
from paper_2108_03409_b300 import stats


def _ar1(rho, T, C, seed):
    rng = np.random.default_rng(seed)
    x = np.empty((T, C))
    x[0] = rng.normal(size=C) / np.sqrt(1 - rho * rho)
    for t in range(1, T):
        x[t] = rho * x[t - 1] + rng.normal(size=C)
    return x


def test_fft_estimator_equals_direct_sum_estimator():
    """Same estimator (full-series mean, Sokal window c = 5) computed by FFT in the package
    and by direct lagged dot products in the oracle: equal to rounding, chain by chain and
    as the chain average, on correlated, white and short series."""
    for rho, T, C in ((0.0, 500, 7), (0.6, 2000, 5), (0.9, 4000, 3), (0.3, 9, 4)):
        x = _ar1(rho, T, C, seed=int(rho * 10) + T)
        for k in range(C):
            a = stats.integrated_autocorr_time(x[:, k])
            b = oracle.tau_int(x[:, k])
            assert abs(a - b) <= 1e-9 * max(1.0, b), (rho, T, k, a, b)
        assert abs(stats.integrated_autocorr_time(x) - oracle.tau_int_chains(x)) <= 1e-9


def test_ar1_closed_form():
    """AR(1) with coefficient rho: rho(t) = rho^t, so tau_int = (1 + rho) / (2 (1 - rho));
    the windowed estimate over 64 chains of 20000 steps is within 5 % of it."""
    for rho in (0.0, 0.5, 0.8):
        ref = (1 + rho) / (2 * (1 - rho))
        got = stats.integrated_autocorr_time(_ar1(rho, 20000, 64, seed=3))
        assert abs(got - ref) <= 0.05 * ref, (rho, got, ref)


def test_constant_and_short_series():
    assert stats.integrated_autocorr_time(np.ones(100)) == 0.5
    assert stats.integrated_autocorr_time(np.arange(3.0)) == 0.5
    assert stats.effective_sample_size(1000, 2.5) == 200.0
