"""Pins of the oracle's lattice code against independent computations.

- Cold start: plaquette and Polyakov loop exactly 1 (Sec. 4).
- Hot start: uniform on S^3 (moments of the Haar measure, Sec. 2).
- Plaquette and Polyakov loop against a brute-force numpy evaluation with 2x2
  complex matrices and np.roll neighbours (independent representation and
  indexing).
- Staple (Sec. 2): replacing one link U by W changes the total sum of
  (1/2) Re Tr U_p over ALL plaquettes (brute force) by exactly
  (1/2) Tr((W - U) V); checked on 2^4, 4^4, 4^3 x 6 and 2^3 x 4.
- Gauge invariance of every per-site plaquette and Polyakov value.
- Unitarity after sweeps, reunitarization, thread-count independence.
"""
import numpy as np
import pytest

import oracle
from test_oracle_primitives import to_matrix

AXIS = {0: 3, 1: 2, 2: 1, 3: 0}  # mu -> axis of the [t, z, y, x] array


def as_matrices(links, ns, nt):
    """links[site, mu, 4] -> complex [t, z, y, x, mu, 2, 2] (float64)."""
    a = links.astype(np.float64).reshape(nt, ns, ns, ns, 4, 4)
    m = np.zeros(a.shape[:-1] + (2, 2), dtype=complex)
    m[..., 0, 0] = a[..., 0] + 1j * a[..., 3]
    m[..., 0, 1] = a[..., 2] + 1j * a[..., 1]
    m[..., 1, 0] = -a[..., 2] + 1j * a[..., 1]
    m[..., 1, 1] = a[..., 0] - 1j * a[..., 3]
    return m


def from_matrices(m, ns, nt):
    a = np.zeros(m.shape[:-2] + (4,), dtype=np.float64)
    a[..., 0] = m[..., 0, 0].real
    a[..., 3] = m[..., 0, 0].imag
    a[..., 2] = m[..., 0, 1].real
    a[..., 1] = m[..., 0, 1].imag
    return a.reshape(ns * ns * ns * nt, 4, 4)


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def shift(m, mu, step=1):
    """Field at x + step*mu."""
    return np.roll(m, -step, axis=AXIS[mu])


def brute_plaquette_sites(links, ns, nt):
    m = as_matrices(links, ns, nt)
    per_site = np.zeros((nt, ns, ns, ns))
    for mu in range(4):
        for nu in range(mu + 1, 4):
            umu = m[..., mu, :, :]
            unu = m[..., nu, :, :]
            p = umu @ shift(unu, mu) @ dag(shift(umu, nu)) @ dag(unu)
            per_site += 0.5 * np.trace(p, axis1=-2, axis2=-1).real
    return per_site.reshape(-1)


def brute_polyakov_sites(links, ns, nt):
    m = as_matrices(links, ns, nt)
    p = m[0, ..., 3, :, :]
    for t in range(1, nt):
        p = p @ m[t, ..., 3, :, :]
    return 0.5 * np.trace(p, axis1=-2, axis2=-1).real.reshape(-1)


def thermal_links(ns, nt, beta, seed, sweeps):
    links = oracle.hot_start(ns, nt, seed)
    for s in range(sweeps):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, links)
    return links


def test_cold_start_observables_are_exactly_one():
    for ns, nt in [(2, 2), (4, 6), (8, 8)]:
        links = oracle.cold_start(ns, nt)
        assert oracle.plaquette(ns, nt, links) == 1.0
        assert oracle.polyakov(ns, nt, links) == 1.0
        assert oracle.plaquette_f64(ns, nt, links) == 1.0


def test_hot_start_is_haar():
    ns, nt = 8, 8
    links = oracle.hot_start(ns, nt, 1)
    a = links.reshape(-1, 4).astype(np.float64)
    n = a.shape[0]
    assert np.abs(np.linalg.norm(a, axis=1) - 1).max() < 1e-6
    # uniform on S^3: E a_i = 0, E a_i a_j = delta_ij / 4, E a_i^4 = 1/8
    sig2 = np.sqrt((1 / 8 - 1 / 16) / n)
    for i in range(4):
        assert abs(a[:, i].mean()) < 5 * 0.5 / np.sqrt(n)
        assert abs((a[:, i] ** 2).mean() - 0.25) < 5 * sig2
        # E a^8 = 105 / (4 6 8 10) on S^3
        assert abs((a[:, i] ** 4).mean() - 1 / 8) < 5 * np.sqrt((105 / 1920 - 1 / 64) / n)
        for j in range(i + 1, 4):
            assert abs((a[:, i] * a[:, j]).mean()) < 5 * 0.25 / np.sqrt(n)
    # hot plaquette: mean of 6V independent-ish traces of Haar elements (var 1/4)
    p = oracle.plaquette(ns, nt, links)
    assert abs(p) < 5 * 0.5 / np.sqrt(6 * ns ** 3 * nt)
    # different seeds give different lattices, same seed the same lattice
    assert not np.array_equal(links, oracle.hot_start(ns, nt, 2))
    assert np.array_equal(links, oracle.hot_start(ns, nt, 1))


@pytest.mark.parametrize("ns,nt", [(2, 2), (4, 6), (6, 4)])
def test_plaquette_and_polyakov_match_brute_force(ns, nt):
    links = thermal_links(ns, nt, 2.3, 7, 3)
    want = brute_plaquette_sites(links, ns, nt)
    got = oracle.site_plaquettes(ns, nt, links)
    assert np.abs(got - want).max() < 4e-6
    assert abs(oracle.plaquette(ns, nt, links) - want.mean() / 6) < 1e-6
    assert abs(oracle.plaquette_f64(ns, nt, links) - want.mean() / 6) < 1e-12
    wantp = brute_polyakov_sites(links, ns, nt)
    assert abs(oracle.polyakov(ns, nt, links) - wantp.mean()) < 2e-6
    assert abs(oracle.polyakov_f64(ns, nt, links) - wantp.mean()) < 1e-12


def total_action_sum(links, ns, nt):
    return brute_plaquette_sites(links, ns, nt).sum()


def qmul64(a, b):
    a0, a1, a2, a3 = a
    b0, b1, b2, b3 = b
    return np.array([a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3,
                     a0 * b1 + a1 * b0 - a2 * b3 + a3 * b2,
                     a0 * b2 + a2 * b0 - a3 * b1 + a1 * b3,
                     a0 * b3 + a3 * b0 - a1 * b2 + a2 * b1])


@pytest.mark.parametrize("ns,nt", [(2, 2), (4, 4), (4, 6), (2, 4)])
def test_staple_is_the_derivative_of_the_action(ns, nt):
    rng = np.random.default_rng(ns * 10 + nt)
    links = oracle.hot_start(ns, nt, 11)
    base = total_action_sum(links, ns, nt)
    vol = ns ** 3 * nt
    for _ in range(12):
        s = int(rng.integers(vol))
        mu = int(rng.integers(4))
        v = oracle.staple(ns, nt, links, s, mu).astype(np.float64)
        w = rng.normal(size=4)
        w /= np.linalg.norm(w)
        old = links[s, mu].astype(np.float64).copy()
        links[s, mu] = w.astype(np.float32)
        changed = total_action_sum(links, ns, nt)
        links[s, mu] = old.astype(np.float32)
        # (1/2) Tr(U V) is component 0 of the quaternion product U V
        w32 = w.astype(np.float32).astype(np.float64)
        want = qmul64(w32, v)[0] - qmul64(old, v)[0]
        assert abs((changed - base) - want) < 2e-5, (s, mu, changed - base, want)
    # matrix form: the staple matrix is to_matrix(v), Tr(U V)/2 real part
    s, mu = 3, 2
    v = oracle.staple(ns, nt, links, s, mu)
    u = links[s, mu]
    assert np.isclose(0.5 * np.trace(to_matrix(u) @ to_matrix(v)).real, qmul64(u.astype(np.float64), v.astype(np.float64))[0])


def random_gauge(ns, nt, rng):
    g = rng.normal(size=(nt, ns, ns, ns, 4))
    g /= np.linalg.norm(g, axis=-1, keepdims=True)
    m = np.zeros(g.shape[:-1] + (2, 2), dtype=complex)
    m[..., 0, 0] = g[..., 0] + 1j * g[..., 3]
    m[..., 0, 1] = g[..., 2] + 1j * g[..., 1]
    m[..., 1, 0] = -g[..., 2] + 1j * g[..., 1]
    m[..., 1, 1] = g[..., 0] - 1j * g[..., 3]
    return m


def test_gauge_invariance_of_observables():
    ns, nt = 4, 6
    links = thermal_links(ns, nt, 2.3, 5, 4)
    rng = np.random.default_rng(9)
    g = random_gauge(ns, nt, rng)
    m = as_matrices(links, ns, nt)
    mt = np.empty_like(m)
    for mu in range(4):
        mt[..., mu, :, :] = g @ m[..., mu, :, :] @ dag(shift(g, mu))
    lt = from_matrices(mt, ns, nt).astype(np.float32)
    assert np.abs(lt - links).max() > 0.1  # the links did change
    p0 = oracle.site_plaquettes(ns, nt, links)
    p1 = oracle.site_plaquettes(ns, nt, lt)
    assert np.abs(p0 - p1).max() < 1e-5
    assert abs(oracle.plaquette(ns, nt, links) - oracle.plaquette(ns, nt, lt)) < 1e-6
    assert abs(oracle.polyakov(ns, nt, links) - oracle.polyakov(ns, nt, lt)) < 2e-6


def test_unitarity_after_sweeps_and_reunitarize():
    ns, nt = 8, 8
    links = oracle.hot_start(ns, nt, 1)
    for s in range(10):
        oracle.heatbath_sweep(ns, nt, 2.3, 1, s, links)
        n = np.linalg.norm(links.reshape(-1, 4).astype(np.float64), axis=1)
        assert np.abs(n - 1).max() <= 1e-6
    rng = np.random.default_rng(2)
    scale = rng.uniform(0.9, 1.1, size=links.shape[:2] + (1,)).astype(np.float32)
    scaled = (links * scale).astype(np.float32)
    oracle.reunitarize(ns, nt, scaled)
    n = np.linalg.norm(scaled.reshape(-1, 4).astype(np.float64), axis=1)
    assert np.abs(n - 1).max() <= 3e-7
    cosang = (scaled.reshape(-1, 4).astype(np.float64) * links.reshape(-1, 4)).sum(1)
    assert np.abs(cosang - 1).max() < 1e-6


def test_threads_do_not_change_the_chain():
    ns, nt = 6, 4
    a = oracle.hot_start(ns, nt, 3)
    b = a.copy()
    ta = [oracle.heatbath_sweep(ns, nt, 2.0, 3, s, a, nthreads=1) for s in range(3)]
    tb = [oracle.heatbath_sweep(ns, nt, 2.0, 3, s, b, nthreads=4) for s in range(3)]
    assert np.array_equal(a, b)
    assert all(np.array_equal(x, y) for x, y in zip(ta, tb))


def test_sweep_is_eight_phases_in_paper_order():
    """Sec. 4: per iteration, even then odd sites for each direction mu before
    the next mu.  Changing the order (odd first) must change the lattice."""
    ns, nt = 4, 4
    a = oracle.hot_start(ns, nt, 4)
    b = a.copy()
    oracle.heatbath_sweep(ns, nt, 2.3, 4, 0, a)
    for mu in range(4):
        for p in (1, 0):
            oracle.heatbath_phase(ns, nt, 2.3, 4, 0, mu, p, b)
    assert not np.array_equal(a, b)
    c = oracle.hot_start(ns, nt, 4)
    for mu in range(4):
        for p in (0, 1):
            oracle.heatbath_phase(ns, nt, 2.3, 4, 0, mu, p, c)
    assert np.array_equal(a, c)
