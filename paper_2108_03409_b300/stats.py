"""Host-side statistics of Markov-chain output: the integrated autocorrelation time of a
scalar series with Sokal's automatic windowing, and the effective sample size."""
from __future__ import annotations

import numpy as np


def integrated_autocorr_time(series: np.ndarray, c: float = 5.0) -> float:
    """tau_int of a [T] series, or the chain average of a [T][C] array.

    rho(t) is the normalised autocovariance estimated with the full-series mean, summed
    from lag 1 until the window W satisfies W >= c * tau(W); tau = 1/2 + sum rho(t)."""
    x = np.asarray(series, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    T = x.shape[0]
    d = x - x.mean(axis=0, keepdims=True)
    # autocovariance of every chain at once through the FFT (zero-padded to 2T)
    f = np.fft.rfft(d, n=2 * T, axis=0)
    acov = np.fft.irfft(f * np.conj(f), axis=0)[:T] / T
    taus = []
    for k in range(x.shape[1]):
        v = acov[0, k]
        if T < 4 or v <= 0:
            taus.append(0.5)
            continue
        tau = 0.5
        for t in range(1, T):
            tau += acov[t, k] / v
            if t >= c * tau:
                break
        taus.append(max(tau, 0.5))
    return float(np.mean(taus))


def effective_sample_size(n: int, tau: float) -> float:
    return n / (2.0 * tau)
