"""Exact reference quantities for the SU(2) heat bath, from the mathematics
(not from the oracle).

The heat-bath density of a0 (Sec. 2) is p(a) = sqrt(1-a^2) exp(x a) / Z(x) on
[-1, 1], x = beta k, with Z(x) = pi I1(x) / x.  With a = cos(theta) the CDF is
F(a) = int_{arccos a}^{pi} sin^2(t) exp(x cos t) dt / Z(x), evaluated here by
Gauss-Legendre quadrature with the factor exp(-x) taken out (scipy's scaled
Bessel function ive) so that large x does not overflow.

Closed forms used by the tests:
  <a0>            = I2(x) / I1(x)
  Creutz accept   = pi I1(x) / (2 sinh x)   (acceptance of sqrt(1-a^2) under the
                    proposal exp(x a) on [-1, 1]); pi/4 in the limit x -> 0
  strong coupling <P> = I2(beta) / I1(beta) to leading order in the character
                    expansion; the first correction is of relative order u^4,
                    u = I2/I1.
"""
import numpy as np
from scipy import optimize, special, stats

_NODES, _WEIGHTS = np.polynomial.legendre.leggauss(400)


def _integral_scaled(theta_lo, x):
    """int_{theta_lo}^{pi} sin^2 t exp(x (cos t - 1)) dt, vectorised in theta_lo."""
    theta_lo = np.atleast_1d(np.asarray(theta_lo, dtype=np.float64))
    half = (np.pi - theta_lo) / 2.0
    mid = (np.pi + theta_lo) / 2.0
    t = mid[:, None] + half[:, None] * _NODES[None, :]
    f = np.sin(t) ** 2 * np.exp(x * (np.cos(t) - 1.0))
    return half * (f @ _WEIGHTS)


def _norm_scaled(x):
    """Z(x) exp(-x) = pi I1(x) exp(-x) / x  (limit pi/2 as x -> 0)."""
    if x < 1e-12:
        return np.pi / 2.0
    return np.pi * special.ive(1, x) / x


def cdf_a0(a, x):
    a = np.clip(np.asarray(a, dtype=np.float64), -1.0, 1.0)
    return _integral_scaled(np.arccos(a), x) / _norm_scaled(x)


def equiprobable_edges(x, nbins=100):
    edges = []
    for j in range(1, nbins):
        target = j / nbins
        edges.append(optimize.brentq(lambda a: cdf_a0(a, x)[0] - target, -1.0, 1.0, xtol=1e-13))
    return np.array(edges)


def chi2_pvalue_a0(samples, x, nbins=100):
    """Pearson chi^2 of samples in nbins equiprobable bins of the exact CDF."""
    edges = equiprobable_edges(x, nbins)
    counts = np.bincount(np.searchsorted(edges, np.asarray(samples, dtype=np.float64)), minlength=nbins)
    expected = len(samples) / nbins
    stat = ((counts - expected) ** 2 / expected).sum()
    return stats.chi2.sf(stat, nbins - 1)


def chi2_pvalue_uniform(samples, lo, hi, nbins=100):
    counts, _ = np.histogram(samples, bins=nbins, range=(lo, hi))
    expected = len(samples) / nbins
    stat = ((counts - expected) ** 2 / expected).sum()
    return stats.chi2.sf(stat, nbins - 1)


def mean_a0(x):
    if x < 1e-12:
        return 0.0
    return special.ive(2, x) / special.ive(1, x)


def creutz_acceptance(x):
    if x < 1e-6:
        return np.pi / 4.0
    # pi I1(x) / (2 sinh x) = pi ive(1,x) / (1 - exp(-2x))
    return np.pi * special.ive(1, x) / (1.0 - np.exp(-2.0 * x))


def strong_coupling_plaquette(beta):
    return special.iv(2, beta) / special.iv(1, beta)
