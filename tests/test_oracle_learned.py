"""Pins of the learned-proposal oracle against mathematics, not itself.

- Spline (Durkan et al. 2019): monotone, f^{-1}(f(z)) = z, the proposal
  density 1/(2 f') integrates to 1 (quadrature), f' equals the central finite
  difference of f.
- -log q and its analytic gradient (implicit differentiation through the
  spline inverse, softmax, softplus, then the MLP) against central finite
  differences in binary64.
- binary32 spline against the binary64 one; MLP against a numpy matrix form.
- Independence Metropolis: a long chain of learned updates of one link with a
  fixed staple has the exact heat-bath law of a0 (Sec. 2), whatever the
  network -- the property that keeps the learned chain exact.
- Collected (beta k, a0) pairs follow the exact conditional law.
"""
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from exact_su2 import cdf_a0, chi2_pvalue_a0, chi2_pvalue_uniform


def random_outputs(rng, scale=1.0):
    return rng.normal(size=25) * scale


def random_weights(rng, scale=0.5, mean=5.0, inv_sd=0.2):
    w = np.zeros(oracle.N_WEIGHTS)
    w[:oracle.N_TRAIN] = rng.normal(size=oracle.N_TRAIN) * scale
    w[oracle.N_TRAIN] = mean
    w[oracle.N_TRAIN + 1] = inv_sd
    return w


def test_spline_binary64_invariants():
    rng = np.random.default_rng(0)
    for _ in range(20):
        o = random_outputs(rng, 2.0)
        zs = np.linspace(-1, 1, 401)
        vals = [oracle.spline_d(o, z) for z in zs]
        a = np.array([v[0] for v in vals])
        assert np.all(np.diff(a) > 0)
        assert abs(a[0] + 1) < 1e-12 and abs(a[-1] - 1) < 1e-12
        assert max(abs(v[2] - z) for v, z in zip(vals, zs)) < 1e-9
        for z in rng.uniform(-0.99, 0.99, 20):
            h = 1e-6
            fd = (oracle.spline_d(o, z + h)[0] - oracle.spline_d(o, z - h)[0]) / (2 * h)
            assert abs(fd - oracle.spline_d(o, z)[1]) < 1e-6 * max(1.0, fd)
        # the proposal density of a0 integrates to one: int_{-1}^{1} exp(-nll(a)) da
        total = integrate.quad(lambda x: np.exp(-oracle.nll_outputs(o, x, False)[0]), -1, 1, limit=200)[0]
        assert abs(total - 1) < 1e-5  # the density has kinks at the knots


def test_nll_output_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    for _ in range(30):
        o = random_outputs(rng, 1.5)
        a = rng.uniform(-0.95, 0.95)
        _, g = oracle.nll_outputs(o, a)
        fd = np.zeros(25)
        for i in range(25):
            d = np.zeros(25)
            d[i] = 1e-6
            fd[i] = (oracle.nll_outputs(o + d, a, False)[0] - oracle.nll_outputs(o - d, a, False)[0]) / 2e-6
        assert np.allclose(g, fd, rtol=1e-5, atol=1e-7), (g, fd)


def test_nll_weight_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    w = random_weights(rng, 0.4)
    pairs = np.stack([rng.uniform(1, 10, 16), rng.uniform(-0.9, 0.95, 16)], axis=1).astype(np.float32)
    val, g = oracle.nll_grad(w, pairs)
    idx = rng.choice(oracle.N_TRAIN, size=120, replace=False)
    for i in idx:
        d = np.zeros_like(w)
        d[i] = 1e-6
        fd = (oracle.nll_grad(w + d, pairs, False)[0] - oracle.nll_grad(w - d, pairs, False)[0]) / 2e-6
        assert abs(g[i] - fd) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, g[i], fd)


def test_binary32_spline_agrees_with_binary64():
    rng = np.random.default_rng(3)
    for _ in range(20):
        o = random_outputs(rng, 1.5).astype(np.float32)
        p = oracle.spline_params(o)
        z = rng.uniform(-1, 1, 2000).astype(np.float32)
        a, fp = oracle.spline_forward(p, z)
        for zi, ai, fi in list(zip(z, a, fp))[:200]:
            a64, f64, _ = oracle.spline_d(o.astype(np.float64), float(zi))
            assert abs(ai - a64) < 3e-5 and abs(fi - f64) < 2e-3 * f64  # binary32 knots (softmax, sums)
        zz, fpi = oracle.spline_inverse(p, a)
        # the inverse is exact up to its conditioning: |dz| f' ~ a few ulp of a
        assert (np.abs(zz - z) * fp).max() < 5e-6
        assert np.allclose(fpi, fp, rtol=5e-3)
        assert np.all(np.diff(a[np.argsort(z)]) >= 0)


def test_mlp_matches_matrix_form():
    rng = np.random.default_rng(4)
    w = random_weights(rng).astype(np.float32)
    W1, b1 = w[0:32].astype(np.float64), w[32:64].astype(np.float64)
    W2, b2 = w[64:1088].reshape(32, 32).astype(np.float64), w[1088:1120].astype(np.float64)
    W3, b3 = w[1120:1920].reshape(25, 32).astype(np.float64), w[1920:1945].astype(np.float64)
    for s in rng.uniform(-3, 3, 50):
        h1 = np.maximum(W1 * np.float32(s) + b1, 0)
        h2 = np.maximum(W2 @ h1 + b2, 0)
        want = W3 @ h2 + b3
        assert np.allclose(oracle.mlp_forward(w, np.float32(s)), want, rtol=1e-5, atol=1e-5)


def test_table_rows_are_the_network_at_grid_points():
    rng = np.random.default_rng(5)
    w = random_weights(rng).astype(np.float32)
    t = oracle.proposal_table(w, -2.0, 3.0, 64)
    ds = np.float32(5.0) / np.float32(63)
    for j in (0, 17, 63):
        s = np.float32(np.float64(j) * np.float64(ds) - 2.0)  # one rounding, as fmaf
        assert np.array_equal(t[j], oracle.spline_params(oracle.mlp_forward(w, s)))
    # interpolation is exact at grid points and monotone knots stay monotone in between
    p = oracle.table_params(t, -2.0, 3.0, 0.123)
    assert np.all(np.diff(p[0:9]) > 0) and np.all(np.diff(p[9:18]) > 0) and np.all(p[18:] > 0)


@pytest.mark.parametrize("bk,scale", [(2.0, 0.3), (8.0, 0.02)])
def test_metropolis_chain_has_the_exact_heatbath_law(bk, scale):
    rng = np.random.default_rng(int(bk * 10))
    w = random_weights(rng, scale, mean=bk, inv_sd=1.0).astype(np.float32)
    table = oracle.proposal_table(w, -1.0, 1.0, 32)
    v = np.array([bk, 0.0, 0.0, 0.0], dtype=np.float32)  # beta = 1: beta k = bk, U~ = 1
    old = np.array([1.0, 0.0, 0.0, 0.0], dtype=np.float32)
    n = 600_000
    a0, acc = oracle.learned_chain(table, -1.0, 1.0, float(w[1945]), float(w[1946]), 1.0, v, old, 99, n)
    assert 0.05 < acc / n <= 1.0
    thin = a0[1000::25].astype(np.float64)
    assert chi2_pvalue_a0(np.clip(thin, -1, 1), bk) > 1e-4


def test_collected_pairs_follow_the_exact_law():
    ns, nt = 8, 8
    links = oracle.hot_start(ns, nt, 3)
    for s in range(5):
        oracle.heatbath_sweep(ns, nt, 2.4, 3, s, links)
    pairs = oracle.collect_pairs(ns, nt, 2.4, 3, 5, 1, 0, 1, links)
    assert pairs.shape[0] == ns ** 3 * nt // 2
    pit = np.array([cdf_a0(a, float(b))[0] for b, a in pairs.astype(np.float64)])
    assert chi2_pvalue_uniform(pit, 0.0, 1.0, nbins=40) > 1e-3
    # the pairs do not move the chain
    before = links.copy()
    oracle.collect_pairs(ns, nt, 2.4, 3, 5, 2, 1, 3, links)
    assert np.array_equal(before, links)


# ------------------------------------------------ the table against the network
# The proposal is defined by the network evaluated at each link's beta k
# (orc_learned_link_net).  The kernel, and orc_learned_link, evaluate the
# network once per grid point of a 256-row table and interpolate every spline
# parameter linearly in s.  The network is piecewise linear in s (ReLU units,
# scalar input) and the spline parameters are smooth functions of its outputs,
# so the interpolation error is O(h^2) between kinks and O(h) in the grid cells
# that hold a kink (h = grid step).  The bounds below are measured on a
# trained network (tests/golden/learned_weights.txt, written from the oracle
# alone) with margin; they make the table a pinned approximation of the
# definition.  Both chains are exact for their own proposal.
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "learned_weights.txt")


def golden_weights():
    with open(GOLDEN) as f:
        w = np.array([float(x) for x in f if not x.startswith("#")], dtype=np.float32)
    assert w.size == oracle.N_WEIGHTS
    return w


def golden_table(G=256, bk_lo=1.0, bk_hi=40.0):
    w = golden_weights()
    mean, scale = w[oracle.N_TRAIN], w[oracle.N_TRAIN + 1]
    s_lo = float(np.float32((bk_lo - mean) * scale))
    s_hi = float(np.float32((bk_hi - mean) * scale))
    return w, oracle.proposal_table(w, s_lo, s_hi, G), s_lo, s_hi


def test_table_parameters_and_density_are_close_to_the_network():
    w, table, s_lo, s_hi = golden_table()
    rng = np.random.default_rng(21)
    h = (s_hi - s_lo) / 255
    ss = np.concatenate([rng.uniform(s_lo, s_hi, 120), s_lo + (np.arange(0, 255, 3) + 0.5) * h]).astype(np.float32)
    a = np.linspace(-1.0, 1.0, 200001)[1:-1].astype(np.float32)
    da = 2.0 / 200000
    z = np.linspace(-1.0, 1.0, 20001)[1:-1].astype(np.float32)
    worst = dict(knot=0.0, der=0.0, tv=0.0, dlogq=0.0)
    for s in ss:
        pt = oracle.table_params(table, s_lo, s_hi, float(s))
        pn = oracle.spline_params(oracle.mlp_forward(w, float(s)))
        worst["knot"] = max(worst["knot"], float(np.abs(pt[:18] - pn[:18]).max()))
        worst["der"] = max(worst["der"], float((np.abs(pt[18:] - pn[18:]) / pn[18:]).max()))
        # total variation between the two proposal densities q = 1 / (2 f'(f^-1(a)))
        _, ft = oracle.spline_inverse(pt, a)
        _, fn = oracle.spline_inverse(pn, a)
        qt, qn = 0.5 / ft.astype(np.float64), 0.5 / fn.astype(np.float64)
        assert abs(qn.sum() * da - 1.0) < 1e-4
        worst["tv"] = max(worst["tv"], 0.5 * float(np.abs(qt - qn).sum()) * da)
        # mean |log q_table - log q_net| over the network's own proposals
        an, fpn = oracle.spline_forward(pn, z)
        _, fpt = oracle.spline_inverse(pt, an)
        worst["dlogq"] = max(worst["dlogq"], float(np.abs(np.log(fpt / fpn.astype(np.float64))).mean()))
    assert worst["knot"] < 3e-3, worst
    assert worst["der"] < 2e-2, worst
    assert worst["tv"] < 4e-3, worst
    assert worst["dlogq"] < 8e-3, worst

@pytest.mark.parametrize("bk", [2.0, 6.0, 12.0, 30.0])
def test_table_acceptance_matches_the_network(bk):
    """Independence-Metropolis chains with the same uniforms, one with the
    table's proposal and one with the network's: acceptances agree within
    2e-3 (the densities differ by at most 4e-3 in total variation)."""
    w, table, s_lo, s_hi = golden_table()
    v = np.array([bk, 0.0, 0.0, 0.0], dtype=np.float32)  # beta = 1: beta k = bk, U~ = 1
    old = np.array([1.0, 0.0, 0.0, 0.0], dtype=np.float32)
    n = 100_000
    mean, scale = float(w[oracle.N_TRAIN]), float(w[oracle.N_TRAIN + 1])
    _, acc_t = oracle.learned_chain(table, s_lo, s_hi, mean, scale, 1.0, v, old, 5, n)
    _, acc_n = oracle.learned_chain_net(w, 1.0, v, old, 5, n)
    assert acc_n / n > 0.85, acc_n / n  # a trained proposal
    assert abs(acc_t - acc_n) / n < 2e-3, (acc_t / n, acc_n / n)


@pytest.mark.parametrize("bk", [3.0, 25.0])
def test_network_chain_has_the_exact_heatbath_law(bk):
    """The proposal as defined (network per step) keeps the heat-bath law."""
    w = golden_weights()
    v = np.array([bk, 0.0, 0.0, 0.0], dtype=np.float32)
    old = np.array([1.0, 0.0, 0.0, 0.0], dtype=np.float32)
    a0, acc = oracle.learned_chain_net(w, 1.0, v, old, 41, 300_000)
    assert acc > 0
    assert chi2_pvalue_a0(np.clip(a0[1000::10].astype(np.float64), -1, 1), bk) > 1e-4


def test_network_sweep_reproduces_the_table_sweep_statistics():
    """A lattice sweep with the network per link and one with the table, from
    the same configuration: acceptances per phase within 0.5% of the links."""
    w, table, s_lo, s_hi = golden_table()
    ns, nt, beta, seed = 6, 6, 2.3, 9
    links = oracle.hot_start(ns, nt, seed)
    for s in range(4):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, links)
    lt, ln = links.copy(), links.copy()
    mean, scale = float(w[oracle.N_TRAIN]), float(w[oracle.N_TRAIN + 1])
    acc_t = oracle.learned_sweep(ns, nt, beta, seed, 4, lt, table, s_lo, s_hi, mean, scale)
    acc_n = oracle.learned_sweep_net(ns, nt, beta, seed, 4, ln, w)
    half = ns ** 3 * nt // 2
    assert np.all(np.abs(acc_t - acc_n) <= 0.005 * half), (acc_t, acc_n)
    assert acc_n.sum() > 0.85 * 8 * half
