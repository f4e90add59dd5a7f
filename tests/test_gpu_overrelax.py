"""GPU parity of the over-relaxation step (the reflection of each link in its
staple, U' = U~^dag U^dag U~^dag): link for link with the oracle on small and
ragged lattices, inside the generation loop (heat bath + n over-relaxation
sweeps), and at 48^4 in the launch configuration the benchmark times; the
action is kept and the map is its own inverse on the device too."""
import os

import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu


def nthreads():
    return min(16, os.cpu_count() or 1)


@pytest.fixture
def made():
    handles = []
    yield handles
    for h in handles:
        su2.su2_destroy(h)


def new_lattice(made, ns, nt, beta, seed, start=su2.SU2_HOT):
    h = su2.su2_create(ns, nt, beta, seed, start)
    made.append(h)
    return h


@pytest.mark.parametrize("ns,nt", [(8, 8), (6, 4), (4, 6), (2, 2), (10, 2)])
def test_phases_link_for_link(made, ns, nt):
    """Every phase on thermalising lattices, including sizes whose V/2 is not
    a multiple of 32 (ragged last round) and the 2^4 extreme."""
    beta, seed = 2.3, 70 + ns
    h = new_lattice(made, ns, nt, beta, seed)
    su2.su2_heatbath_sweep(h, 2)
    ref = su2.su2_get_links(h, ns, nt)
    for mu in range(4):
        for parity in range(2):
            su2.su2_overrelax_phase(h, mu, parity)
            oracle.overrelax_phase(ns, nt, mu, parity, ref)
            assert np.array_equal(su2.su2_get_links(h, ns, nt), ref), (mu, parity)


def test_generate_with_overrelaxation_matches_oracle(made):
    """su2_set_overrelax(2): each heat-bath sweep is followed by two
    over-relaxation sweeps; links, plaquettes and counters as the oracle's."""
    ns, nt, beta, seed = 8, 8, 2.3, 1
    h = new_lattice(made, ns, nt, beta, seed)
    su2.su2_set_overrelax(h, 2)
    plaq, poly, st = su2.su2_generate(h, 5, 1, 0)
    ref = oracle.hot_start(ns, nt, seed)
    for s in range(5):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, ref, nthreads=nthreads())
        oracle.overrelax_sweep(ns, nt, ref)
        oracle.overrelax_sweep(ns, nt, ref)
        want = oracle.plaquette(ns, nt, ref)
        assert abs(plaq[s] - want) <= 1e-6 * max(abs(want), 0.05), s
    assert np.array_equal(su2.su2_get_links(h, ns, nt), ref)
    assert st["sweeps"] == 5 and st["overrelax_sweeps"] == 10
    assert st["overrelax_updates"] == 10 * 4 * ns ** 3 * nt
    # the heat-bath counter advanced by the heat-bath sweeps only
    assert su2.su2_get_state(h)["sweep"] == 5
    # switched off again: plain heat bath
    su2.su2_set_overrelax(h, 0)
    su2.su2_heatbath_sweep(h, 1)
    oracle.heatbath_sweep(ns, nt, beta, seed, 5, ref, nthreads=nthreads())
    assert np.array_equal(su2.su2_get_links(h, ns, nt), ref)


def test_involution_and_kept_action_on_device(made):
    ns, nt = 16, 16
    h = new_lattice(made, ns, nt, 2.5, 9)
    su2.su2_heatbath_sweep(h, 3)
    before = su2.su2_get_links(h, ns, nt)
    p0 = su2.su2_plaquette(h)
    su2.su2_overrelax_phase(h, 2, 1)
    moved = su2.su2_get_links(h, ns, nt)
    assert abs(su2.su2_plaquette(h) - p0) < 2e-7
    assert np.abs(moved - before).max() > 0.1
    su2.su2_overrelax_phase(h, 2, 1)
    assert np.abs(su2.su2_get_links(h, ns, nt) - before).max() < 2e-6
    su2.su2_overrelax_sweep(h, 4)
    assert abs(su2.su2_plaquette(h) - p0) < 2e-6


def test_timing_and_arguments(made):
    h = new_lattice(made, 8, 4, 2.3, 3)
    su2.su2_set_timing(h, True)
    su2.su2_set_overrelax(h, 3)
    st = su2.su2_heatbath_sweep(h, 2, stats=True)
    assert st["timed"] and st["kernel_ms"] > 0 and st["overrelax_ms"] > 0
    assert st["overrelax_sweeps"] == 6
    for bad in ((-1,), (65,)):
        with pytest.raises(su2.SU2Error):
            su2.su2_set_overrelax(h, *bad)
    for mu, parity in ((4, 0), (-1, 0), (0, 2)):
        with pytest.raises(su2.SU2Error):
            su2.su2_overrelax_phase(h, mu, parity)
    with pytest.raises(su2.SU2Error):
        su2.su2_overrelax_sweep(h, -1)


def test_full_size_48(made):
    """48^4 at beta = 6 after two heat-bath sweeps from the hot start: one
    over-relaxation sweep, whole lattice against the oracle."""
    ns = nt = 48
    h = new_lattice(made, ns, nt, 6.0, 3)
    su2.su2_heatbath_sweep(h, 2)
    ref = su2.su2_get_links(h, ns, nt)
    p0 = oracle.plaquette(ns, nt, ref)
    su2.su2_overrelax_sweep(h, 1)
    oracle.overrelax_sweep(ns, nt, ref, nthreads=nthreads())
    assert np.array_equal(su2.su2_get_links(h, ns, nt), ref)
    assert abs(su2.su2_plaquette(h) - p0) < 1e-6
