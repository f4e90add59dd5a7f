"""Statistical pins of the oracle's heat bath (Sec. 2) against exact results.

- a0 draws at fixed beta k: chi^2 in 100 equiprobable bins of the exact CDF of
  sqrt(1-a^2) exp(beta k a); mean a0 = I2/I1; mean number of Creutz trials =
  1 / (pi I1(x) / (2 sinh x)).
- A link updated many times inside a fixed lattice: (1/2) Tr(U'V)/k follows the
  same exact law, and the direction of the vector part is uniform on S^2.
- Strong coupling: <P> = I2(beta)/I1(beta) for beta <= 0.5.
- beta = 0: one sweep gives Haar-distributed links.
- The tau_int estimator on an AR(1) series with known tau_int.
"""
import numpy as np
from scipy import stats
import pytest

import oracle
from exact_su2 import (chi2_pvalue_a0, chi2_pvalue_uniform, creutz_acceptance, mean_a0,
                       strong_coupling_plaquette)
from paper_1010_1486_gb300.analysis import tau_int

N_DRAWS = 1_000_000


@pytest.mark.parametrize("bk", [1e-7, 0.5, 2.0, 5.0, 15.0, 36.0])
def test_a0_sampler_exact_distribution(bk):
    a0, trials = oracle.creutz_a0_many(bk, seed=20 + int(bk * 10), n=N_DRAWS)
    assert trials.min() >= 1
    assert np.all(np.abs(a0) <= 1.0)
    p = chi2_pvalue_a0(a0.astype(np.float64), float(np.float32(bk)))
    assert p > 1e-3, p
    # mean a0 = I2/I1 within 5 sigma
    m = a0.astype(np.float64).mean()
    sd = a0.astype(np.float64).std() / np.sqrt(N_DRAWS)
    assert abs(m - mean_a0(float(np.float32(bk)))) < 5 * sd
    # mean trials of a geometric law with success probability = acceptance
    acc = creutz_acceptance(float(np.float32(bk)))
    mt = trials.mean()
    sdt = np.sqrt((1 - acc) / acc ** 2 / N_DRAWS)
    assert abs(mt - 1 / acc) < 5 * sdt, (mt, 1 / acc)


def test_creutz_acceptance_values_quoted_for_the_workloads():
    # beta k ~ 0.5 (strong coupling), 5, 30 (beta = 6 ordered lattice)
    assert abs(creutz_acceptance(0.5) - 0.78) < 0.01
    assert abs(creutz_acceptance(5.0) - 0.52) < 0.01
    assert abs(creutz_acceptance(30.0) - 0.23) < 0.01


def test_heatbath_link_conditional_on_a_lattice():
    ns, nt = 4, 4
    links = oracle.hot_start(ns, nt, 31)
    for s in range(3):
        oracle.heatbath_sweep(ns, nt, 2.3, 31, s, links)
    site, mu = 37, 2
    beta = 2.3
    v = oracle.staple(ns, nt, links, site, mu)
    par = sum(int(c) for c in np.unravel_index(site, (nt, ns, ns, ns))) & 1
    out, trials = oracle.heatbath_link_many(beta, v, seed=31, eo=site >> 1, parity=par, mu=mu, n=N_DRAWS, sweep0=1000)
    assert trials.min() >= 1
    u = out.astype(np.float64)
    vd = v.astype(np.float64)
    k = np.sqrt((vd ** 2).sum())
    bk = float(np.float32(beta) * np.float32(k))
    # U' V / k = a  (the heat-bath variable), computed in binary64
    a = np.stack([u[:, 0] * vd[0] - u[:, 1] * vd[1] - u[:, 2] * vd[2] - u[:, 3] * vd[3],
                  u[:, 0] * vd[1] + u[:, 1] * vd[0] - u[:, 2] * vd[3] + u[:, 3] * vd[2],
                  u[:, 0] * vd[2] + u[:, 2] * vd[0] - u[:, 3] * vd[1] + u[:, 1] * vd[3],
                  u[:, 0] * vd[3] + u[:, 3] * vd[0] - u[:, 1] * vd[2] + u[:, 2] * vd[1]], axis=1) / k
    assert np.abs(np.linalg.norm(u, axis=1) - 1).max() < 1e-6
    assert chi2_pvalue_a0(np.clip(a[:, 0], -1, 1), bk) > 1e-3
    r = np.linalg.norm(a[:, 1:], axis=1)
    keep = r > 1e-3
    c = a[keep, 3] / r[keep]
    phi = np.arctan2(a[keep, 2], a[keep, 1])
    assert chi2_pvalue_uniform(c, -1.0, 1.0) > 1e-3
    assert chi2_pvalue_uniform(phi, -np.pi, np.pi) > 1e-3
    # independence of a0 and the direction: a0 in its lower / upper half gives the same c law
    med = np.median(a[keep, 0])
    lo = c[a[keep, 0] < med]
    hi = c[a[keep, 0] >= med]
    assert abs(lo.mean() - hi.mean()) < 5 * np.sqrt(2 / 3 / len(lo))


@pytest.mark.parametrize("beta", [0.1, 0.25, 0.5])
def test_strong_coupling_plaquette(beta):
    ns, nt = 6, 6
    therm, meas = 20, 1500
    seed = int(beta * 1000) + 7
    links = oracle.hot_start(ns, nt, seed)
    series = []
    for s in range(therm + meas):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, links, nthreads=min(8, oracle.max_threads()))
        if s >= therm:
            series.append(oracle.plaquette(ns, nt, links))
    series = np.array(series)
    tau, _, _, err = tau_int(series)
    want = strong_coupling_plaquette(beta)
    u = want
    # next order of the character expansion is O(u^5) (cubes): 4 u^5 as a bound
    tol = max(4 * err, 2e-4) + 4 * u ** 5
    assert abs(series.mean() - want) < tol, (series.mean(), want, err, tau)


def test_beta_zero_sweep_gives_haar_links():
    ns, nt = 8, 8
    links = oracle.cold_start(ns, nt)
    oracle.heatbath_sweep(ns, nt, 0.0, 77, 0, links)
    a = links.reshape(-1, 4).astype(np.float64)
    n = a.shape[0]
    assert abs(a[:, 0].mean()) < 5 * 0.5 / np.sqrt(n)
    assert abs((a[:, 0] ** 2).mean() - 0.25) < 5 * np.sqrt(1 / 16 / n)
    assert chi2_pvalue_a0(a[:, 0], 0.0) > 1e-3
    assert abs(oracle.plaquette(ns, nt, links)) < 5 * 0.5 / np.sqrt(6 * ns ** 3 * nt)


def test_tau_int_on_ar1_series():
    rng = np.random.default_rng(5)
    rho = 0.9
    n = 400_000
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - rho ** 2)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + e[i]
    tau, dtau, w, err = tau_int(x)
    want = (1 + rho) / (2 * (1 - rho))
    assert abs(tau - want) < max(3 * dtau, 0.05 * want), (tau, dtau, want)
    # the same chain cut into 16 replicas of 25,000: pooled estimate agrees
    tau_r, dtau_r, _, _ = tau_int([x[i * 25_000:(i + 1) * 25_000] for i in range(16)])
    assert abs(tau_r - want) < max(3 * dtau_r, 0.06 * want), (tau_r, want)
    # short replicas: pooled estimate stays close where averaging per-run estimates is biased low/high
    reps = [x[i * 250:(i + 1) * 250] for i in range(16)]
    tau_s, dtau_s, _, _ = tau_int(reps)
    assert abs(tau_s - want) < 0.35 * want, (tau_s, want)
    # replicas taken along a drifting chain: each about its own mean, the
    # drift between replicas stays out of tau
    drift = [x[i * 2_000:(i + 1) * 2_000] + 3.0 * i for i in range(16)]
    tau_d, dtau_d, _, _ = tau_int(drift, own_means=True)
    assert abs(tau_d - want) < max(3 * dtau_d, 0.1 * want), (tau_d, want)
    assert tau_int(drift)[0] > 2 * want  # about the common mean the drift looks like correlation
    # white noise: tau = 1/2
    tau0, _, _, err0 = tau_int(rng.normal(size=100_000))
    assert abs(tau0 - 0.5) < 0.05
    assert abs(err0 - 1 / np.sqrt(100_000)) < 0.1 / np.sqrt(100_000)


# ------------------------------------------------- Kennedy-Pendleton sampler
@pytest.mark.parametrize("bk", [2.0, 5.0, 15.0, 36.0])
def test_kennedy_pendleton_exact_distribution(bk):
    a0, trials = oracle.kp_a0_many(bk, seed=77 + int(bk), n=N_DRAWS)
    assert trials.min() >= 1
    assert chi2_pvalue_a0(a0.astype(np.float64), float(np.float32(bk))) > 1e-3
    m = a0.astype(np.float64).mean()
    sd = a0.astype(np.float64).std() / np.sqrt(N_DRAWS)
    assert abs(m - mean_a0(float(np.float32(bk)))) < 5 * sd
    # far fewer trials than Creutz's method where beta k is large
    if bk >= 15:
        assert trials.mean() < 1.1 and trials.mean() < 0.5 / creutz_acceptance(bk)


def test_kennedy_pendleton_chain_matches_creutz_chain():
    """Both samplers draw the same heat-bath law: equal <P> at beta = 2.3."""
    ns, nt, beta = 6, 6, 2.3
    res = []
    for sweep_fn, seed in ((oracle.heatbath_sweep, 41), (oracle.heatbath_sweep_kp, 42)):
        links = oracle.hot_start(ns, nt, seed)
        series = []
        for s in range(1200):
            sweep_fn(ns, nt, beta, seed, s, links, nthreads=min(8, oracle.max_threads()))
            if s >= 200:
                series.append(oracle.plaquette(ns, nt, links))
        series = np.array(series)
        _, _, _, err = tau_int(series)
        res.append((series.mean(), err))
    (m1, e1), (m2, e2) = res
    assert abs(m1 - m2) < 4 * np.hypot(e1, e2), res


def _direction(out, ut):
    """(c, phi) of the vector part of a = U' U~ (U' = a U~^dag): a3 = r c,
    (a1, a2) = r sqrt(1 - c^2) (cos phi, sin phi)."""
    a = oracle.quat_mul(out, ut)
    r = np.sqrt(max(1.0 - float(a[0]) ** 2, 1e-30))
    return float(a[3]) / r, float(np.arctan2(a[2], a[1])) % (2 * np.pi)


def test_paired_links_draw_independent_uniform_directions():
    """The two links of a pair (even/odd indices 2j, 2j + 1) take their
    direction uniforms from different words of one Philox block: each
    direction is uniform on the sphere (c uniform in [-1, 1], phi in
    [0, 2 pi)) and the pair's directions are independent (2-D chi^2 on
    (c_even, c_odd), (phi_even, phi_odd) and (c_even, phi_odd))."""
    v = np.array([2.1, -0.7, 0.4, 1.3], dtype=np.float32)
    k = float(np.sqrt(np.dot(v.astype(np.float64), v)))
    ut = np.array([v[0] / k, v[1] / k, v[2] / k, v[3] / k], dtype=np.float32)  # U~ = V / k
    n = 12_000
    ce, co, pe, po = np.empty(n), np.empty(n), np.empty(n), np.empty(n)
    for j in range(n):
        a, _ = oracle.heatbath_link(1.5, v, 77, 2 * j, 3, 1, 2)
        b, _ = oracle.heatbath_link(1.5, v, 77, 2 * j + 1, 3, 1, 2)
        ce[j], pe[j] = _direction(a, ut)
        co[j], po[j] = _direction(b, ut)
    for x, lo, hi in ((ce, -1, 1), (co, -1, 1), (pe, 0, 2 * np.pi), (po, 0, 2 * np.pi)):
        assert chi2_pvalue_uniform(x, lo, hi, nbins=40) > 1e-3
    for x, y, xr, yr in ((ce, co, (-1, 1), (-1, 1)), (pe, po, (0, 2 * np.pi), (0, 2 * np.pi)),
                         (ce, po, (-1, 1), (0, 2 * np.pi))):
        h, _, _ = np.histogram2d(x, y, bins=8, range=(xr, yr))
        e = n / 64.0
        assert stats.chi2.sf(((h - e) ** 2 / e).sum(), 63) > 1e-3
    assert np.corrcoef(ce, co)[0, 1] ** 2 < 1e-3
