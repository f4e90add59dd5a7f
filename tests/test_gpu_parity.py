"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

The heat bath is an exact Markov chain driven by counter-based random
numbers, and both sides follow the same binary32 arithmetic contract, so the
bar is link-for-link agreement (max |da| <= 2e-5, expected 0) with identical
per-phase trial counts, and plaquette / Polyakov loop within 1e-6 relative.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu

LINK_TOL = 2e-5
OBS_REL = 1e-6


def obs_close(got, want, scale=0.05):
    return abs(got - want) <= OBS_REL * max(abs(want), scale)


def nthreads():
    return min(16, os.cpu_count() or 1)


class Lattice:
    def __init__(self, ns, nt, beta, seed, start):
        self.ns, self.nt = ns, nt
        self.h = su2.su2_create(ns, nt, beta, seed, start)

    def close(self):
        if self.h:
            su2.su2_destroy(self.h)
            self.h = None

    def links(self):
        return su2.su2_get_links(self.h, self.ns, self.nt)


@pytest.fixture
def lattice():
    made = []

    def make(ns, nt, beta, seed, start=su2.SU2_HOT):
        lat = Lattice(ns, nt, beta, seed, start)
        made.append(lat)
        return lat

    yield make
    for lat in made:
        lat.close()


# ------------------------------------------------------------ building blocks
def test_philox_matches_oracle():
    rng = np.random.default_rng(0)
    ck = rng.integers(0, 2 ** 32, size=(4096, 6), dtype=np.uint64).astype(np.uint32)
    ck[0] = 0
    ck[1] = 0xFFFFFFFF
    got = su2.su2_selftest_philox(ck)
    for row, g in zip(ck, got):
        want = oracle.philox4x32_10(row[2:], row[:2])
        assert np.array_equal(g, want)


def test_elementary_functions_bitwise():
    rng = np.random.default_rng(1)
    x = rng.integers(0x00800000, 0x3F800001, size=1_000_000, dtype=np.uint32).view(np.float32)
    assert np.array_equal(su2.su2_selftest_math(0, x).view(np.uint32), oracle.logf(x).view(np.uint32))
    y = rng.uniform(-87.0, 0.0, size=1_000_000).astype(np.float32)
    assert np.array_equal(su2.su2_selftest_math(1, y).view(np.uint32), oracle.expf(y).view(np.uint32))
    u = (np.arange(1, 2 ** 24 + 1, dtype=np.float64) * 2.0 ** -24).astype(np.float32)
    s, c = su2.su2_selftest_math(2, u)
    so, co = oracle.sincos2pi(u)
    assert np.array_equal(s.view(np.uint32), so.view(np.uint32))
    assert np.array_equal(c.view(np.uint32), co.view(np.uint32))


def test_creutz_trial_variable_matches_definition_over_beta_k():
    """x = e + r1 (1 - e) and the candidate a0 of a Creutz trial, device
    against oracle, bitwise, over beta k in [16, 44] (through the kernels'
    exp(-2 beta k) cutoff at 21 and the definition's at 43) for every word
    below 2^16 (the smallest log uniforms, from 2^-33) and random words."""
    rng = np.random.default_rng(7)
    words = np.concatenate([np.arange(0, 1 << 16), rng.integers(0, 2 ** 32, 8192),
                            np.arange(2 ** 32 - 256, 2 ** 32)]).astype(np.uint32)
    bks = np.concatenate([np.linspace(16.0, 44.0, 113), [17.0, 17.5, 20.5, 21.0, 43.0],
                          [np.nextafter(np.float32(21.0), np.float32(50.0)),
                           np.nextafter(np.float32(43.0), np.float32(50.0))]]).astype(np.float32)
    bk = np.repeat(bks, words.size).astype(np.float32)
    w = np.tile(words, bks.size)
    x_ref, a0_ref = oracle.creutz_x_a0(bk, w)
    q = np.stack([bk, w.view(np.float32)], axis=1)
    x, a0 = su2.su2_selftest_math(6, q)
    assert np.array_equal(x.view(np.uint32), x_ref.view(np.uint32))
    assert np.array_equal(a0.view(np.uint32), a0_ref.view(np.uint32))


# ------------------------------------------------------------- start kernels
@pytest.mark.parametrize("ns,nt", [(2, 2), (4, 6), (6, 4), (8, 8), (12, 4)])
def test_starts_match_oracle(lattice, ns, nt):
    cold = lattice(ns, nt, 2.3, 5, su2.SU2_COLD)
    assert np.array_equal(cold.links(), oracle.cold_start(ns, nt))
    assert su2.su2_plaquette(cold.h) == 1.0
    assert su2.su2_polyakov(cold.h) == 1.0
    hot = lattice(ns, nt, 2.3, 5, su2.SU2_HOT)
    assert np.array_equal(hot.links(), oracle.hot_start(ns, nt, 5))


def test_set_get_links_roundtrip(lattice):
    ns, nt = 6, 4
    lat = lattice(ns, nt, 2.0, 3)
    rng = np.random.default_rng(3)
    links = rng.normal(size=(ns ** 3 * nt, 4, 4)).astype(np.float32)
    su2.su2_set_links(lat.h, links)
    assert np.array_equal(lat.links(), links)


@pytest.mark.parametrize("ns,nt", [(6, 4), (2, 2), (16, 8)])
def test_links_through_pinned_host_memory(lattice, ns, nt):
    """Page-locked host buffers are read and written by the layout kernel
    directly; the result equals the staged path for pageable buffers."""
    import torch

    lat = lattice(ns, nt, 2.0, 4)
    su2.su2_heatbath_sweep(lat.h, 1)
    pageable = lat.links()
    pinned = torch.empty((ns ** 3 * nt, 4, 4), dtype=torch.float32, pin_memory=True).numpy()
    su2.su2_get_links(lat.h, ns, nt, out=pinned)
    assert np.array_equal(pinned, pageable)
    rng = np.random.default_rng(5)
    pinned[...] = rng.normal(size=pinned.shape).astype(np.float32)
    su2.su2_set_links(lat.h, pinned)
    assert np.array_equal(lat.links(), pinned)


# -------------------------------------------------------------- sweep parity
def run_parity(lattice, ns, nt, beta, seed, start, sweeps):
    lat = lattice(ns, nt, beta, seed, start)
    ref = oracle.hot_start(ns, nt, seed) if start == su2.SU2_HOT else oracle.cold_start(ns, nt)
    for s in range(sweeps):
        st = su2.su2_heatbath_sweep(lat.h, 1, stats=True)
        tr = oracle.heatbath_sweep(ns, nt, beta, seed, s, ref, nthreads=nthreads())
        got = lat.links()
        d = float(np.abs(got - ref).max())
        assert d <= LINK_TOL, (s, d)
        assert st["trials"] == [int(t) for t in tr], (s, st["trials"], list(tr))
        assert st["sampler_failures"] == 0
        assert st["link_updates"] == 4 * ns ** 3 * nt
        p, l = su2.su2_plaquette(lat.h), su2.su2_polyakov(lat.h)
        assert obs_close(p, oracle.plaquette(ns, nt, ref)), (s, p)
        assert obs_close(l, oracle.polyakov(ns, nt, ref)), (s, l)
    return lat, ref


def test_plain_8x8x8x8_ten_sweeps_link_for_link(lattice):
    """8^4, beta = 2.3, hot start from seed 1, 10 sweeps, plaquette after each."""
    lat, ref = run_parity(lattice, 8, 8, 2.3, 1, su2.SU2_HOT, 10)
    assert np.array_equal(lat.links(), ref)  # the contract makes them bitwise equal


@pytest.mark.parametrize("ns,nt,beta", [(2, 2, 2.3), (4, 4, 1.7), (6, 4, 2.5), (4, 6, 2.2), (12, 4, 2.4),
                                        (2, 8, 3.0), (10, 2, 2.0)])
def test_index_coverage_and_ragged_tails(lattice, ns, nt, beta):
    # 6^3x4: V/2 = 432 is not a multiple of the block size; 2^4 wraps onto itself
    run_parity(lattice, ns, nt, beta, 11 + ns + nt, su2.SU2_HOT, 3)


@pytest.mark.parametrize("beta", [0.0, 0.25, 60.0])
def test_degenerate_couplings(lattice, beta):
    # beta = 0: Haar branch; beta = 60 on a cold lattice: beta k > 43 (exp -> 0)
    run_parity(lattice, 4, 4, beta, 21, su2.SU2_COLD, 2)
    run_parity(lattice, 4, 4, beta, 22, su2.SU2_HOT, 2)


def test_zero_sweeps_is_a_no_op(lattice):
    lat = lattice(4, 4, 2.3, 1)
    before = lat.links()
    st = su2.su2_heatbath_sweep(lat.h, 0, stats=True)
    assert st["sweeps"] == 0 and st["trials"] == [0] * 8
    assert np.array_equal(before, lat.links())
    assert su2.su2_get_state(lat.h)["sweep"] == 0


def test_single_phase_matches_oracle(lattice):
    ns, nt, beta, seed = 6, 6, 2.3, 4
    lat = lattice(ns, nt, beta, seed)
    ref = oracle.hot_start(ns, nt, seed)
    for mu in range(4):
        for p in range(2):
            su2.su2_heatbath_phase(lat.h, mu, p)
            oracle.heatbath_phase(ns, nt, beta, seed, 0, mu, p, ref)
            assert np.array_equal(lat.links(), ref), (mu, p)


def test_generate_measures_and_reunitarizes_like_the_oracle(lattice):
    ns, nt, beta, seed = 6, 6, 2.5, 2
    lat = lattice(ns, nt, beta, seed, su2.SU2_COLD)
    plaq, poly, st = su2.su2_generate(lat.h, 12, measure_every=1, reunit_every=5)
    ref = oracle.cold_start(ns, nt)
    for s in range(12):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, ref)
        if (s + 1) % 5 == 0:
            oracle.reunitarize(ns, nt, ref)
        assert obs_close(plaq[s], oracle.plaquette(ns, nt, ref)), s
        assert obs_close(poly[s], oracle.polyakov(ns, nt, ref)), s
    assert np.array_equal(lat.links(), ref)
    assert st["sweeps"] == 12 and st["kernel_launches"] == 96


def test_reunitarize_matches_oracle(lattice):
    ns, nt = 4, 4
    lat = lattice(ns, nt, 2.3, 9)
    rng = np.random.default_rng(9)
    links = lat.links() * rng.uniform(0.5, 1.5, size=(ns ** 3 * nt, 4, 1)).astype(np.float32)
    links = links.astype(np.float32)
    su2.su2_set_links(lat.h, links)
    su2.su2_reunitarize(lat.h)
    oracle.reunitarize(ns, nt, links)
    assert np.array_equal(lat.links(), links)


def test_resume_is_bitwise(lattice):
    ns, nt, beta, seed = 6, 4, 2.3, 8
    a = lattice(ns, nt, beta, seed)
    su2.su2_heatbath_sweep(a.h, 10)
    full = a.links()
    b = lattice(ns, nt, beta, seed)
    su2.su2_heatbath_sweep(b.h, 5)
    saved_links, saved_state = b.links(), su2.su2_get_state(b.h)
    c = lattice(ns, nt, 1.0, 999, su2.SU2_COLD)
    su2.su2_set_links(c.h, saved_links)
    su2.su2_set_state(c.h, saved_state)
    su2.su2_heatbath_sweep(c.h, 5)
    assert np.array_equal(c.links(), full)


def test_timing_reports_each_phase_kernel(lattice):
    lat = lattice(8, 8, 2.3, 1)
    su2.su2_set_timing(lat.h, True)
    st = su2.su2_heatbath_sweep(lat.h, 3, stats=True)
    assert st["timed"] and st["kernel_ms"] > 0 and st["kernel_launches"] == 24


def test_bad_phase_arguments(lattice):
    lat = lattice(4, 4, 2.3, 1)
    for mu, p in [(-1, 0), (4, 0), (0, 2)]:
        with pytest.raises(su2.SU2Error):
            su2.su2_heatbath_phase(lat.h, mu, p)
    with pytest.raises(su2.SU2Error):
        su2.su2_set_state(lat.h, {"ns": 6, "nt": 4, "beta": 1.0, "seed": 1, "sweep": 0})


def test_torch_allocator_and_stream():
    torch = pytest.importorskip("torch")
    su2.use_torch_allocator()
    try:
        stream = torch.cuda.Stream()
        h = su2.su2_create(4, 4, 2.3, 1, su2.SU2_HOT, stream=stream)
        try:
            su2.su2_heatbath_sweep(h, 2)
            got = su2.su2_get_links(h, 4, 4)
        finally:
            su2.su2_destroy(h)
        ref = oracle.hot_start(4, 4, 1)
        for s in range(2):
            oracle.heatbath_sweep(4, 4, 2.3, 1, s, ref)
        assert np.array_equal(got, ref)
    finally:
        su2.use_default_allocator()


# ------------------------------------------------- full size (48^4, beta = 6)
def test_full_size_48_hot_start_one_sweep(lattice):
    """48^4, beta = 6.0, hot start from seed 3: the launch configuration the
    benchmark times.  Whole lattice compared bit for bit after the start and
    after each of two sweeps (the first from the hot start puts many links
    at 17 < beta k < 21, the second more above; the oracle runs threaded
    over sites)."""
    ns = nt = 48
    beta, seed = 6.0, 3
    lat = lattice(ns, nt, beta, seed)
    ref = oracle.hot_start(ns, nt, seed)
    assert np.array_equal(lat.links(), ref)
    for s in range(2):
        st = su2.su2_heatbath_sweep(lat.h, 1, stats=True)
        tr = oracle.heatbath_sweep(ns, nt, beta, seed, s, ref, nthreads=nthreads())
        assert np.array_equal(lat.links(), ref), s
        assert st["trials"] == [int(t) for t in tr], s
    assert obs_close(su2.su2_plaquette(lat.h), oracle.plaquette(ns, nt, ref))
    assert obs_close(su2.su2_polyakov(lat.h), oracle.polyakov(ns, nt, ref))


def test_benchmark_path_full_size_48():
    """The benchmark's own path: the PyTorch allocator, a lattice on a user
    stream, the Kennedy-Pendleton sampler, su2_generate measuring every sweep
    (warm-up sweeps capture the sweep's CUDA graph, the next ones replay it).
    After 3 + 2 sweeps from the hot start the whole 48^4 lattice is bitwise
    the oracle's, and each sweep's plaquette (fused into the sweep) and
    Polyakov loop agree with the oracle's within 1e-6."""
    torch = pytest.importorskip("torch")
    ns = nt = 48
    beta, seed = 6.0, 3
    su2.use_torch_allocator()
    try:
        stream = torch.cuda.Stream()
        h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT, stream=stream)
        try:
            su2.su2_set_sampler(h, su2.SU2_SAMPLER_KP)
            p_w, l_w, _ = su2.su2_generate(h, 3, 1, 0)
            p_t, l_t, st = su2.su2_generate(h, 2, 1, 0)
            got = su2.su2_get_links(h, ns, nt)
        finally:
            su2.su2_destroy(h)
    finally:
        su2.use_default_allocator()
    plaq, poly = list(p_w) + list(p_t), list(l_w) + list(l_t)
    ref = oracle.hot_start(ns, nt, seed)
    for s in range(5):
        oracle.heatbath_sweep_kp(ns, nt, beta, seed, s, ref, nthreads=nthreads())
        assert obs_close(plaq[s], oracle.plaquette(ns, nt, ref)), s
        assert obs_close(poly[s], oracle.polyakov(ns, nt, ref)), s
    assert np.array_equal(got, ref)
    assert st["link_updates"] == 2 * 4 * ns ** 3 * nt


# ------------------------------------------------ Kennedy-Pendleton sampler
@pytest.mark.parametrize("ns,nt,beta,start", [(8, 8, 2.3, su2.SU2_HOT), (6, 4, 6.0, su2.SU2_HOT),
                                              (4, 6, 0.4, su2.SU2_COLD), (12, 4, 2.5, su2.SU2_COLD)])
def test_kennedy_pendleton_sweeps_link_for_link(lattice, ns, nt, beta, start):
    seed = 60 + ns
    lat = lattice(ns, nt, beta, seed, start)
    su2.su2_set_sampler(lat.h, su2.SU2_SAMPLER_KP)
    ref = oracle.hot_start(ns, nt, seed) if start == su2.SU2_HOT else oracle.cold_start(ns, nt)
    for s in range(4):
        st = su2.su2_heatbath_sweep(lat.h, 1, stats=True)
        tr = oracle.heatbath_sweep_kp(ns, nt, beta, seed, s, ref, nthreads=nthreads())
        assert st["trials"] == [int(t) for t in tr], s
        assert np.array_equal(lat.links(), ref), s
    assert obs_close(su2.su2_plaquette(lat.h), oracle.plaquette(ns, nt, ref))


def test_kennedy_pendleton_full_size_48(lattice):
    ns = nt = 48
    lat = lattice(ns, nt, 6.0, 3)
    su2.su2_heatbath_sweep(lat.h, 2)
    ref = lat.links()
    su2.su2_set_sampler(lat.h, su2.SU2_SAMPLER_KP)
    st = su2.su2_heatbath_sweep(lat.h, 1, stats=True)
    tr = oracle.heatbath_sweep_kp(ns, nt, 6.0, 3, 2, ref, nthreads=nthreads())
    assert st["trials"] == [int(t) for t in tr]
    assert np.array_equal(lat.links(), ref)
    # about one trial per link at beta = 6
    assert sum(tr) / (4 * ns ** 3 * nt) < 1.2
