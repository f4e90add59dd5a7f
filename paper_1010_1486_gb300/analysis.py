"""Host-side statistics for Monte Carlo time series.

Integrated autocorrelation time by the Gamma method with automatic windowing
(U. Wolff, "Monte Carlo errors with less errors", Comput. Phys. Commun. 156
(2004) 143; window rule of Madras & Sokal, J. Stat. Phys. 50 (1988) 109 refined
by Wolff's S parameter).  Convention: tau_int = 1/2 + sum_{t>=1} rho(t), so an
uncorrelated series has tau_int = 1/2 and the error of the mean is
sqrt(2 tau_int Gamma(0) / N).
"""
from __future__ import annotations

import math

import numpy as np


def autocorrelation(series: np.ndarray, tmax: int) -> np.ndarray:
    """Gamma(t) for t = 0..tmax, normalised by N - t, via FFT."""
    a = np.asarray(series, dtype=np.float64)
    n = a.size
    d = a - a.mean()
    nfft = 1 << (2 * n - 1).bit_length()
    f = np.fft.rfft(d, nfft)
    acf = np.fft.irfft(f * np.conj(f), nfft)[: tmax + 1]
    return acf / (n - np.arange(tmax + 1))


def _pooled_autocovariance(replicas, tmax: int, own_means: bool = False) -> np.ndarray:
    """Gamma(t), t = 0..tmax, of several runs of the same chain (replicas):
    deviations from the common mean (or, with own_means, from each run's own
    mean, which keeps a slow drift between runs out of Gamma), lag products
    summed over all runs, divided by the number of pairs (Wolff 2004,
    Sec. 3.3)."""
    mean = np.concatenate(replicas).mean()
    num = np.zeros(tmax + 1)
    pairs = np.zeros(tmax + 1)
    for a in replicas:
        n = a.size
        d = a - (a.mean() if own_means else mean)
        nfft = 1 << (2 * n - 1).bit_length()
        f = np.fft.rfft(d, nfft)
        acf = np.fft.irfft(f * np.conj(f), nfft)
        m = min(tmax, n - 1)
        num[: m + 1] += acf[: m + 1]
        pairs[: m + 1] += n - np.arange(m + 1)
    return num / np.maximum(pairs, 1.0)


def tau_int(series, s_factor: float = 1.5, own_means: bool = False):
    """Returns (tau_int, its statistical error, window W, error of the mean).
    `series` is one run, or a list of runs of the same chain (replicas: their
    autocovariances are pooled before the windowed sum, which avoids the bias
    of averaging tau_int over short runs; about the common mean, or with
    own_means about each run's mean, for runs taken at different times of a
    slowly drifting chain)."""
    if isinstance(series, (list, tuple)):
        replicas = [np.asarray(r, dtype=np.float64) for r in series]
    else:
        replicas = [np.asarray(series, dtype=np.float64)]
    n = sum(r.size for r in replicas)
    if min(r.size for r in replicas) < 4:
        raise ValueError("series too short")
    tmax = min(min(r.size for r in replicas) // 2, 100000)
    gamma = (autocorrelation(replicas[0], tmax) if len(replicas) == 1
             else _pooled_autocovariance(replicas, tmax, own_means))
    if gamma[0] <= 0.0:
        return 0.5, 0.0, 0, 0.0
    rho = gamma / gamma[0]
    cum = 0.5 + np.cumsum(rho[1:])  # tau_int(W) for W = 1..tmax
    window = tmax
    for w in range(1, tmax + 1):
        t = cum[w - 1]
        if t <= 0.5:
            tau_w = 1e-12
        else:
            tau_w = s_factor / math.log((2.0 * t + 1.0) / (2.0 * t - 1.0))
        g = math.exp(-w / tau_w) - tau_w / math.sqrt(w * n)
        if g < 0.0:
            window = w
            break
    # bias correction of Gamma(0) and of the summed autocorrelation (Wolff, Eq. 49)
    cf = gamma[0] + 2.0 * gamma[1: window + 1].sum()
    cf *= 1.0 + (2.0 * window + 1.0) / n
    g0 = gamma[0] + cf / n  # corrected variance estimate
    tau = max(0.5 * cf / g0, 0.5)
    dtau = tau * math.sqrt(2.0 * (2.0 * window + 1.0) / n)
    err_mean = math.sqrt(max(cf, 0.0) / n)
    return tau, dtau, window, err_mean


def interleaved_offset(test_means, ref_means, position: float):
    """Offset of one form against a reference form from interleaved blocks:
    block k of the test form runs between reference blocks k and k + 1, its
    centre `position` (0..1) of the way from the centre of reference block k
    to that of block k + 1.  Each test block is compared with the reference
    interpolated linearly at its centre, so a slow linear drift of the chain
    cancels (the midpoint of the two reference blocks would leave a bias of
    (position - 1/2) times the drift per round).  Returns (mean offset, its
    standard error from the spread of the per-block offsets)."""
    t = np.asarray(test_means, dtype=np.float64)
    r = np.asarray(ref_means, dtype=np.float64)
    if r.size != t.size + 1 or t.size < 2:
        raise ValueError("need n >= 2 test blocks and n + 1 reference blocks")
    d = t - (r[:-1] + position * (r[1:] - r[:-1]))
    return float(d.mean()), float(d.std(ddof=1) / math.sqrt(d.size))


def block_drift(block_means):
    """Linear drift of a chain's block means b_k (k = 0..n-1, one block per
    round of interleaved blocks): least-squares slope per round, its standard
    error, and the scatter of one block mean about the line (its error).
    A chain in equilibrium has |slope| well below that block error."""
    b = np.asarray(block_means, dtype=np.float64)
    n = b.size
    if n < 3:
        raise ValueError("need at least 3 blocks")
    k = np.arange(n, dtype=np.float64)
    kc = k - k.mean()
    slope = float((kc * (b - b.mean())).sum() / (kc * kc).sum())
    resid = b - (b.mean() + slope * kc)
    block_err = float(math.sqrt((resid * resid).sum() / (n - 2)))
    slope_err = block_err / math.sqrt(float((kc * kc).sum()))
    return slope, slope_err, block_err


def effective_potential(w) -> np.ndarray:
    """Static-potential estimates from Wilson loops W[R-1, T-1]:
    V_eff(R, T) = log(W(R, T) / W(R, T+1)), shape (rmax, tmax - 1).  For large
    T, W(R, T) ~ C(R) exp(-V(R) T), so V_eff(R, T) -> V(R) (NaN unless both
    loops are positive)."""
    w = np.asarray(w, dtype=np.float64)
    ok = (w[:, :-1] > 0) & (w[:, 1:] > 0)
    a = np.where(ok, w[:, :-1], 1.0)
    b = np.where(ok, w[:, 1:], 1.0)
    return np.where(ok, np.log(a / b), np.nan)


def cornell_fit(r, v):
    """Least-squares fit V(R) = V0 - alpha/R + sigma R; returns (V0, alpha, sigma)."""
    r = np.asarray(r, dtype=np.float64)
    a = np.stack([np.ones_like(r), -1.0 / r, r], axis=1)
    coef, *_ = np.linalg.lstsq(a, np.asarray(v, dtype=np.float64), rcond=None)
    return tuple(float(c) for c in coef)
