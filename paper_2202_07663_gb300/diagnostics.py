"""Convergence diagnostics of MCMC samples (arXiv:2202.07663, Sec. 2.5).

- ``autocorr``: the empirical autocorrelation of one chain as the paper
  defines it (Sec. 2.5.2, after Sokal 1996):
  rho(tau) = c(tau)/c(0), c(tau) = 1/(N - tau) sum_{n <= N - tau} (f_n - mu)(f_{n+tau} - mu).
- ``ess``: effective sample size of several chains, N_total / tau with
  rho averaged over chains and the sum truncated by Geyer's initial positive
  sequence. Default: tau = 1 + 2 sum_{k>=0} (rho(2k+1) + rho(2k+2)) over the
  leading positive pairs, so ESS <= N_total (a negative lag-1 correlation is
  cut, as in a truncation at the first negative autocorrelation).
  ``antithetic=True``: Geyer's own form, tau = -1 + 2 sum_{k>=0}
  (rho(2k) + rho(2k+1)) over the leading positive pairs, which exceeds
  N_total for anti-correlated chains.
- ``rhat``: the potential scale reduction factor of Gelman & Rubin (1992):
  sqrt(((n-1)/n W + B/n) / W), W the mean within-chain variance, B/n the
  variance of the chain means.
Samples are arrays [chains, draws] (or [chains, draws, d], diagnosed per
column).
"""
from __future__ import annotations

import numpy as np


def autocorr(x: np.ndarray, max_lag: int | None = None) -> np.ndarray:
    x = np.asarray(x, np.float64)
    N = x.shape[-1]
    L = N - 1 if max_lag is None else min(max_lag, N - 1)
    d = x - x.mean(axis=-1, keepdims=True)
    # c(tau) for all lags by FFT, normalised by N - tau
    n2 = 1 << int(np.ceil(np.log2(2 * N)))
    f = np.fft.rfft(d, n=n2, axis=-1)
    acov = np.fft.irfft(f * np.conj(f), n=n2, axis=-1)[..., : L + 1]
    acov = acov / (N - np.arange(L + 1))
    return acov / acov[..., :1]


def _ess_1d(chains: np.ndarray, antithetic: bool) -> float:
    m, n = chains.shape
    rho = autocorr(chains).mean(axis=0)
    s = 0.0
    k = 0
    off = 0 if antithetic else 1
    while 2 * k + 1 + off < n:
        pair = rho[2 * k + off] + rho[2 * k + 1 + off]
        if pair <= 0:
            break
        s += pair
        k += 1
    tau = (-1.0 + 2.0 * s) if antithetic else (1.0 + 2.0 * s)
    return m * n / tau


def ess(samples: np.ndarray, antithetic: bool = False) -> np.ndarray:
    s = np.asarray(samples, np.float64)
    if s.ndim == 2:
        return np.array(_ess_1d(s, antithetic))
    return np.array([_ess_1d(s[:, :, j], antithetic) for j in range(s.shape[2])])


def rhat(samples: np.ndarray) -> np.ndarray:
    s = np.asarray(samples, np.float64)
    n = s.shape[1]
    means = s.mean(axis=1)
    W = s.var(axis=1, ddof=1).mean(axis=0)
    B_over_n = means.var(axis=0, ddof=1)
    var_plus = (n - 1) / n * W + B_over_n
    return np.sqrt(var_plus / W)
