"""Pins of the oracle's over-relaxation step (the reflection that keeps the
local action of a link, the usual companion of the Sec. 2 heat bath).

- the quaternion result against the 2x2 complex-matrix formula
  U' = W^dag U^dag W^dag, W = V/|V|, in binary64 (fixes the order of the
  products and every conjugation), and Re Tr U'V = Re Tr UV;
- applied twice it gives the link back; |U'| = 1;
- on a lattice: one phase (or a sweep) leaves the mean plaquette unchanged
  while moving the links, and touches no link outside the phase;
- heat bath + over-relaxation samples the same <P> as the heat bath alone.
"""
import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300.analysis import tau_int

SIGMA = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]], complex),
         np.array([[1, 0], [0, -1]], complex)]


def to_matrix(a):
    a = np.asarray(a, dtype=np.float64)
    return a[0] * np.eye(2) + 1j * sum(a[j + 1] * SIGMA[j] for j in range(3))


def from_matrix(m):
    return np.array([np.trace(m).real / 2] + [(np.trace(m @ SIGMA[j]) / 2j).real for j in range(3)])


def random_unit(rng, n):
    a = rng.normal(size=(n, 4))
    return (a / np.linalg.norm(a, axis=1, keepdims=True)).astype(np.float32)


def test_quaternion_algebra_matches_matrices():
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=4), rng.normal(size=4)
    got = np.zeros(4, np.float32)
    lib = oracle._load()
    aa, bb = a.astype(np.float32), b.astype(np.float32)
    lib.orc_quat_mul(oracle._ptr(aa), oracle._ptr(bb), oracle._ptr(got))
    want = from_matrix(to_matrix(aa) @ to_matrix(bb))
    assert np.allclose(got, want, atol=1e-6)


def test_overrelax_link_matches_matrix_reflection():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        u = random_unit(rng, 1)[0]
        v = (rng.normal(size=4) * rng.uniform(0.1, 6.0)).astype(np.float32)
        got = oracle.overrelax_link(v, u).astype(np.float64)
        w = to_matrix(v) / np.linalg.norm(v.astype(np.float64))
        um = to_matrix(u)
        want = from_matrix(w.conj().T @ um.conj().T @ w.conj().T)
        assert np.abs(got - want).max() < 2e-6, (got, want)
        # the action term is kept, the link itself moves
        vm = to_matrix(v)
        before = np.trace(um @ vm).real
        after = np.trace(to_matrix(got) @ vm).real
        assert abs(after - before) < 4e-6 * np.linalg.norm(v), (before, after)
        assert abs(np.linalg.norm(got) - 1) < 1e-6


def test_overrelax_zero_staple_is_the_inverse():
    u = np.array([0.5, -0.5, 0.5, 0.5], np.float32)
    assert np.array_equal(oracle.overrelax_link(np.zeros(4, np.float32), u), np.array([0.5, 0.5, -0.5, -0.5], np.float32))


def test_overrelax_is_an_involution():
    rng = np.random.default_rng(8)
    for _ in range(2000):
        u = random_unit(rng, 1)[0]
        v = (rng.normal(size=4) * 3).astype(np.float32)
        back = oracle.overrelax_link(v, oracle.overrelax_link(v, u))
        assert np.abs(back - u).max() < 2e-6


@pytest.mark.parametrize("mu,parity", [(0, 0), (2, 1), (3, 0)])
def test_overrelax_phase_keeps_the_action(mu, parity):
    ns, nt = 4, 6
    links = oracle.hot_start(ns, nt, 21)
    for s in range(3):
        oracle.heatbath_sweep(ns, nt, 2.3, 21, s, links)
    before = links.copy()
    p0 = oracle.plaquette(ns, nt, links)
    oracle.overrelax_phase(ns, nt, mu, parity, links)
    p1 = oracle.plaquette(ns, nt, links)
    assert abs(p1 - p0) < 3e-7, (p0, p1)
    # exactly the links of the phase changed
    sites = np.arange(ns ** 3 * nt)
    c = np.stack(np.unravel_index(sites, (nt, ns, ns, ns)))
    par = c.sum(axis=0) & 1
    moved = np.abs(links - before).max(axis=2)  # [site, mu]
    mask = np.zeros_like(moved, dtype=bool)
    mask[par == parity, mu] = True
    assert np.all(moved[~mask] == 0)
    assert moved[mask].min() > 0 and moved[mask].max() > 0.1


def test_overrelax_sweep_keeps_the_action():
    ns, nt = 6, 4
    links = oracle.hot_start(ns, nt, 22)
    for s in range(5):
        oracle.heatbath_sweep(ns, nt, 2.5, 22, s, links)
    p0 = oracle.plaquette(ns, nt, links)
    for _ in range(3):
        oracle.overrelax_sweep(ns, nt, links)
    assert abs(oracle.plaquette(ns, nt, links) - p0) < 1e-6


def test_heatbath_with_overrelaxation_samples_the_same_plaquette():
    ns, nt, beta = 6, 6, 2.3
    nth = min(8, oracle.max_threads())
    res = []
    for n_or, seed in ((0, 51), (2, 52)):
        links = oracle.hot_start(ns, nt, seed)
        series = []
        for s in range(1200):
            oracle.heatbath_sweep(ns, nt, beta, seed, s, links, nthreads=nth)
            for _ in range(n_or):
                oracle.overrelax_sweep(ns, nt, links, nthreads=nth)
            if s >= 200:
                series.append(oracle.plaquette(ns, nt, links))
        series = np.array(series)
        tau, _, _, err = tau_int(series)
        res.append((series.mean(), err, tau))
    (m1, e1, _), (m2, e2, _) = res
    assert abs(m1 - m2) < 4 * np.hypot(e1, e2), res
