"""Pins of the oracle's space-time Wilson loops W(R, T).

- cold start: every loop is 1;
- single loops against a complex-matrix walk around the rectangle in
  binary64 (x -> x+Ri -> x+Ri+Tt -> x+Tt -> x), including loops that wrap;
- W(1, 1) against the space-time plaquette computed independently in numpy;
- gauge invariance under a random gauge transformation;
- strong coupling: W(1,1) = u, W(1,2) = W(2,1) = u^2 to leading order,
  u = I2(beta)/I1(beta), at beta = 0.5.
"""
import numpy as np
import pytest

import oracle
from exact_su2 import strong_coupling_plaquette
from paper_1010_1486_gb300.analysis import tau_int

SIGMA = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]], complex),
         np.array([[1, 0], [0, -1]], complex)]


def mats(links):
    a = links.astype(np.float64)
    return (a[..., 0, None, None] * np.eye(2) + 1j * sum(a[..., j + 1, None, None] * SIGMA[j] for j in range(3)))


def coords(site, ns, nt):
    t, z, y, x = np.unravel_index(site, (nt, ns, ns, ns))
    return [int(x), int(y), int(z), int(t)]


def index(c, ns, nt):
    return ((c[3] % nt) * ns + c[2] % ns) * ns * ns + (c[1] % ns) * ns + c[0] % ns


def walk(m, ns, nt, site, i, R, T):
    c = coords(site, ns, nt)
    prod = np.eye(2, dtype=complex)
    for _ in range(R):
        prod = prod @ m[index(c, ns, nt), i]
        c[i] += 1
    for _ in range(T):
        prod = prod @ m[index(c, ns, nt), 3]
        c[3] += 1
    for _ in range(R):
        c[i] -= 1
        prod = prod @ m[index(c, ns, nt), i].conj().T
    for _ in range(T):
        c[3] -= 1
        prod = prod @ m[index(c, ns, nt), 3].conj().T
    return np.trace(prod).real / 2


def test_cold_start_loops_are_one():
    links = oracle.cold_start(4, 6)
    assert np.array_equal(oracle.wilson_loops(4, 6, links, 4, 6), np.ones((4, 6)))


@pytest.mark.parametrize("ns,nt", [(4, 6), (6, 4)])
def test_single_loops_against_matrix_walk(ns, nt):
    links = oracle.hot_start(ns, nt, 5)
    oracle.heatbath_sweep(ns, nt, 1.5, 5, 0, links)
    m = mats(links)
    rng = np.random.default_rng(3)
    for _ in range(300):
        site = int(rng.integers(ns ** 3 * nt))
        i = int(rng.integers(3))
        R, T = int(rng.integers(1, ns + 1)), int(rng.integers(1, nt + 1))
        got = oracle.wilson_loop_at(ns, nt, links, site, i, R, T)
        assert abs(got - walk(m, ns, nt, site, i, R, T)) < 2e-6, (site, i, R, T)


def test_w11_is_the_space_time_plaquette():
    ns, nt = 4, 4
    links = oracle.hot_start(ns, nt, 6)
    oracle.heatbath_sweep(ns, nt, 2.0, 6, 0, links)
    m = mats(links)
    acc = 0.0
    for site in range(ns ** 3 * nt):
        c = coords(site, ns, nt)
        for i in range(3):
            ci = c.copy(); ci[i] += 1
            ct = c.copy(); ct[3] += 1
            p = m[site, i] @ m[index(ci, ns, nt), 3] @ m[index(ct, ns, nt), i].conj().T @ m[site, 3].conj().T
            acc += np.trace(p).real / 2
    want = acc / (3 * ns ** 3 * nt)
    assert abs(oracle.wilson_loops(ns, nt, links, 1, 1)[0, 0] - want) < 1e-6


def test_gauge_invariance():
    ns, nt = 4, 6
    links = oracle.hot_start(ns, nt, 7)
    oracle.heatbath_sweep(ns, nt, 2.3, 7, 0, links)
    w0 = oracle.wilson_loops(ns, nt, links, 3, 3)
    rng = np.random.default_rng(9)
    g = rng.normal(size=(ns ** 3 * nt, 4))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    gm = mats(g.astype(np.float32))
    m = mats(links)
    out = np.empty_like(links)
    for site in range(ns ** 3 * nt):
        c = coords(site, ns, nt)
        for mu in range(4):
            cm = c.copy(); cm[mu] += 1
            u = gm[site] @ m[site, mu] @ gm[index(cm, ns, nt)].conj().T
            out[site, mu] = [np.trace(u).real / 2] + [(np.trace(u @ SIGMA[j]) / 2j).real for j in range(3)]
    w1 = oracle.wilson_loops(ns, nt, out, 3, 3)
    assert np.abs(w1 - w0).max() < 3e-6, np.abs(w1 - w0).max()
    assert np.abs(w0).max() > 1e-3  # not trivially zero


def test_strong_coupling_area_law():
    ns, nt, beta, seed = 6, 6, 0.5, 11
    u = strong_coupling_plaquette(beta)
    links = oracle.hot_start(ns, nt, seed)
    nth = min(8, oracle.max_threads())
    w = []
    for s in range(420):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, links, nthreads=nth)
        if s >= 20:
            w.append(oracle.wilson_loops(ns, nt, links, 2, 2, nthreads=nth))
    w = np.array(w)
    for (R, T), area in (((1, 1), 1), ((1, 2), 2), ((2, 1), 2)):
        series = w[:, R - 1, T - 1]
        _, _, _, err = tau_int(series)
        assert abs(series.mean() - u ** area) < 4 * err + 4 * u ** (area + 4), (R, T, series.mean(), u ** area, err)
