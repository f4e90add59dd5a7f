"""Learned proposal on the GPU against the CPU oracle: the proposal table
(network evaluated at grid points), learned Metropolis sweeps with the plain
heat bath as fallback, and the collection of (beta k, a0) training pairs --
all link for link / bit for bit, through the C ABI."""
import os

import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu


def threads():
    return min(16, os.cpu_count() or 1)


def weights(seed, scale=0.3, mean=4.0, inv_sd=0.5):
    rng = np.random.default_rng(seed)
    w = np.zeros(su2.N_WEIGHTS, dtype=np.float32)
    w[:1945] = rng.normal(size=1945) * scale
    w[1945], w[1946] = mean, inv_sd
    return w


def test_proposal_table_is_bitwise_the_oracles():
    h = su2.su2_create(4, 4, 2.3, 1, su2.SU2_HOT)
    try:
        for seed, (lo, hi, G) in enumerate([(-3.0, 3.0, 256), (-1.5, 2.5, 64), (0.0, 1.0, 2)]):
            w = weights(seed, 0.5)
            su2.su2_set_proposal(h, w, lo, hi, G)
            got = su2.su2_get_proposal_table(h, G)
            want = oracle.proposal_table(w, lo, hi, G)
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), seed
    finally:
        su2.su2_destroy(h)


@pytest.mark.parametrize("ns,nt,beta", [(4, 4, 2.3), (6, 4, 1.8), (8, 8, 2.4)])
def test_learned_sweeps_link_for_link(ns, nt, beta):
    seed = 41
    w = weights(ns + nt, 0.2, mean=beta * 3.0, inv_sd=0.6)
    lo, hi, G = -3.0, 3.0, 128
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT)
    try:
        su2.su2_heatbath_sweep(h, 2)
        su2.su2_set_proposal(h, w, lo, hi, G)
        plaq, poly, st = su2.su2_learned_generate(h, 3, 1, 0.0)
        got = su2.su2_get_links(h, ns, nt)
    finally:
        su2.su2_destroy(h)
    links = oracle.hot_start(ns, nt, seed)
    for s in range(2):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, links)
    table = oracle.proposal_table(w, lo, hi, G)
    acc = np.zeros(8, dtype=np.int64)
    for s in range(2, 5):
        acc += oracle.learned_sweep(ns, nt, beta, seed, s, links, table, lo, hi, float(w[1945]), float(w[1946]))
        assert abs(plaq[s - 2] - oracle.plaquette(ns, nt, links)) <= 1e-6 * max(1, abs(plaq[s - 2]))
    assert np.array_equal(got, links)
    assert st["accepted"] == [int(a) for a in acc]
    assert st["learned_sweeps"] == 3 and st["plain_sweeps"] == 0
    assert 0 < sum(acc) < 3 * 4 * ns ** 3 * nt


def test_fallback_alternates_with_the_plain_heat_bath():
    ns, nt, beta, seed = 6, 6, 2.3, 5
    w = weights(9, 0.2, mean=7.0, inv_sd=0.5)
    lo, hi, G = -3.0, 3.0, 64
    threshold = 0.999  # no learned sweep reaches it: every learned sweep is followed by a plain one
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT)
    try:
        su2.su2_set_proposal(h, w, lo, hi, G)
        _, _, st = su2.su2_learned_generate(h, 5, 0, threshold)
        got = su2.su2_get_links(h, ns, nt)
    finally:
        su2.su2_destroy(h)
    links = oracle.hot_start(ns, nt, seed)
    table = oracle.proposal_table(w, lo, hi, G)
    learned = True
    n_learned = n_plain = 0
    acc_total = np.zeros(8, dtype=np.int64)
    trials = np.zeros(8, dtype=np.int64)
    for s in range(5):
        if learned:
            acc = oracle.learned_sweep(ns, nt, beta, seed, s, links, table, lo, hi, float(w[1945]), float(w[1946]))
            acc_total += acc
            n_learned += 1
            learned = not (acc.sum() < threshold * 4 * ns ** 3 * nt)
        else:
            trials += oracle.heatbath_sweep(ns, nt, beta, seed, s, links)
            n_plain += 1
            learned = True
    assert np.array_equal(got, links)
    assert (st["learned_sweeps"], st["plain_sweeps"]) == (n_learned, n_plain) == (3, 2)
    assert st["accepted"] == [int(a) for a in acc_total]
    assert st["plain_trials"] == [int(t) for t in trials]


def test_collected_pairs_are_bitwise_the_oracles():
    torch = pytest.importorskip("torch")
    ns, nt, beta, seed = 8, 6, 2.4, 12
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT)
    try:
        su2.su2_heatbath_sweep(h, 3)
        links = su2.su2_get_links(h, ns, nt)
        buf = torch.zeros((ns ** 3 * nt, 2), dtype=torch.float32, device="cuda")
        for mu, par, stride in [(0, 0, 1), (3, 1, 5), (2, 0, 7)]:
            n = su2.su2_collect_pairs(h, mu, par, stride, buf.data_ptr(), buf.shape[0])
            torch.cuda.synchronize()
            got = buf[:n].cpu().numpy()
            want = oracle.collect_pairs(ns, nt, beta, seed, 3, mu, par, stride, links)
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (mu, par, stride)
        assert np.array_equal(su2.su2_get_links(h, ns, nt), links)  # the chain did not move
    finally:
        su2.su2_destroy(h)


def test_learned_sweep_with_the_cpu_trained_network_matches_the_oracle():
    """su2_learned_sweep (fallback at 0.7, no measurements) with the network
    that the oracle trained on exact draws (tests/golden/learned_weights.txt):
    the kernel chain is bitwise the oracle's table chain, with equal
    acceptance counts, and its acceptance is that of the network's own chain
    within the table's pinned error."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "learned_weights.txt")
    with open(path) as f:
        w = np.array([float(x) for x in f if not x.startswith("#")], dtype=np.float32)
    mean, scale = float(w[1945]), float(w[1946])
    lo, hi = float(np.float32((1.0 - mean) * scale)), float(np.float32((40.0 - mean) * scale))
    ns, nt, beta, seed = 8, 8, 2.4, 17
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT)
    try:
        su2.su2_heatbath_sweep(h, 3)
        su2.su2_set_proposal(h, w, lo, hi, 256)
        st = su2.su2_learned_sweep(h, 2)
        got = su2.su2_get_links(h, ns, nt)
    finally:
        su2.su2_destroy(h)
    assert st["plain_sweeps"] == 0 and st["learned_sweeps"] == 2
    links = oracle.hot_start(ns, nt, seed)
    for s in range(3):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, links)
    start = links.copy()
    table = oracle.proposal_table(w, lo, hi, 256)
    acc = np.zeros(8, dtype=np.int64)
    for s in range(3, 5):
        acc += oracle.learned_sweep(ns, nt, beta, seed, s, links, table, lo, hi, mean, scale)
    assert np.array_equal(got, links)
    assert [int(a) for a in st["accepted"]] == [int(a) for a in acc]
    net = np.zeros(8, dtype=np.int64)
    for s in range(3, 5):
        net += oracle.learned_sweep_net(ns, nt, beta, seed, s, start, w)
    half = ns ** 3 * nt // 2
    assert abs(int(acc.sum()) - int(net.sum())) <= 0.005 * 16 * half, (acc, net)
    assert acc.sum() > 0.85 * 16 * half


def test_learned_sweep_full_size_48():
    """One learned sweep of the benchmark's 48^4, beta = 6 lattice from its
    hot start, in the benchmark's launch configuration, with the network the
    oracle trained (tests/golden/learned_weights.txt): bitwise the oracle's
    table chain over all 21 million links, with equal acceptance counts."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "learned_weights.txt")
    with open(path) as f:
        w = np.array([float(x) for x in f if not x.startswith("#")], dtype=np.float32)
    mean, scale = float(w[1945]), float(w[1946])
    lo, hi = float(np.float32((1.0 - mean) * scale)), float(np.float32((40.0 - mean) * scale))
    ns = nt = 48
    beta, seed = 6.0, 3
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT)
    try:
        su2.su2_set_proposal(h, w, lo, hi, 256)
        st = su2.su2_learned_sweep(h, 1)
        got = su2.su2_get_links(h, ns, nt)
    finally:
        su2.su2_destroy(h)
    assert st["learned_sweeps"] == 1 and st["plain_sweeps"] == 0
    links = oracle.hot_start(ns, nt, seed)
    table = oracle.proposal_table(w, lo, hi, 256)
    acc = oracle.learned_sweep(ns, nt, beta, seed, 0, links, table, lo, hi, mean, scale)
    assert np.array_equal(got, links)
    assert [int(a) for a in st["accepted"]] == [int(a) for a in acc]
    assert acc.sum() > 0.85 * 4 * ns ** 3 * nt


@pytest.mark.parametrize("min_acceptance", [0.7, 0.999])
def test_graph_replayed_learned_sweeps_equal_eager_sweeps(min_acceptance):
    """su2_learned_generate on a lattice with a stream replays each sweep
    (learned phases, gated plain phases, fallback decision, measurement) from
    a CUDA graph; the chain, the acceptance counts, the fallback alternation
    (forced at min_acceptance 0.999) and the measurements equal the eager
    path's bit for bit."""
    torch = pytest.importorskip("torch")
    ns, nt, beta, seed = 8, 8, 2.4, 23
    w = weights(7, 0.2, mean=beta * 3.0, inv_sd=0.6)
    out = []
    for stream in (None, torch.cuda.Stream()):
        h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT, stream=stream)
        try:
            su2.su2_heatbath_sweep(h, 2)
            su2.su2_set_proposal(h, w, -3.0, 3.0, 128)
            plaq, poly, st = su2.su2_learned_generate(h, 6, 2, min_acceptance)
            plaq2, poly2, st2 = su2.su2_learned_generate(h, 3, 1, min_acceptance)
            out.append((su2.su2_get_links(h, ns, nt), plaq.copy(), poly.copy(), st, plaq2.copy(), st2))
        finally:
            su2.su2_destroy(h)
    (l0, p0, q0, s0, r0, t0), (l1, p1, q1, s1, r1, t1) = out
    assert np.array_equal(l0, l1)
    assert np.array_equal(p0, p1) and np.array_equal(q0, q1) and np.array_equal(r0, r1)
    for a, b in ((s0, s1), (t0, t1)):
        assert a["accepted"] == b["accepted"]
        assert a["learned_sweeps"] == b["learned_sweeps"] and a["plain_sweeps"] == b["plain_sweeps"]
    if min_acceptance > 0.9:
        assert s0["plain_sweeps"] > 0
