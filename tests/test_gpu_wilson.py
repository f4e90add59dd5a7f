"""GPU Wilson loops against the oracle: every (R, T) up to the lattice
extents (loops that wrap included), on small, ragged and 24^4 lattices.  Each
loop is the same binary32 computation on both sides; only the binary64 sum
order differs."""
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


@pytest.mark.parametrize("ns,nt,rmax,tmax,beta,sweeps", [(8, 8, 4, 4, 2.3, 3), (6, 4, 6, 4, 2.0, 2),
                                                          (4, 6, 2, 6, 1.0, 1), (2, 2, 2, 2, 2.3, 1),
                                                          (8, 4, 8, 3, 5.0, 2)])
def test_loops_match_oracle(made, ns, nt, rmax, tmax, beta, sweeps):
    h = su2.su2_create(ns, nt, beta, 40 + ns, su2.SU2_HOT)
    made.append(h)
    su2.su2_heatbath_sweep(h, sweeps)
    links = su2.su2_get_links(h, ns, nt)
    got = su2.su2_wilson_loops(h, rmax, tmax)
    want = oracle.wilson_loops(ns, nt, links, rmax, tmax, nthreads=nthreads())
    assert np.abs(got - want).max() < 1e-12, np.abs(got - want).max()


def test_cold_start_and_24x24x24x24(made):
    h = su2.su2_create(24, 24, 2.5, 2, su2.SU2_COLD)
    made.append(h)
    assert np.array_equal(su2.su2_wilson_loops(h, 5, 5), np.ones((5, 5)))
    su2.su2_heatbath_sweep(h, 40)
    links = su2.su2_get_links(h, 24, 24)
    got = su2.su2_wilson_loops(h, 4, 4)
    want = oracle.wilson_loops(24, 24, links, 4, 4, nthreads=nthreads())
    assert np.abs(got - want).max() < 1e-12
    # area-law shape: W falls with R and with T
    assert np.all(np.diff(got, axis=0) < 0) and np.all(np.diff(got, axis=1) < 0)
    # repeated calls give the same bits
    assert np.array_equal(su2.su2_wilson_loops(h, 4, 4), got)


def test_bad_extents(made):
    h = su2.su2_create(6, 4, 2.3, 1, su2.SU2_HOT)
    made.append(h)
    for rmax, tmax in ((0, 1), (1, 0), (7, 1), (1, 5), (17, 1)):
        with pytest.raises(su2.SU2Error):
            su2.su2_wilson_loops(h, rmax, tmax)


def test_static_potential_rises_with_distance(made):
    """Confinement at beta = 2.5 on 16^4: the effective potential from
    W(R, T) / W(R, T+1) grows with R."""
    from paper_1010_1486_gb300.analysis import effective_potential

    h = su2.su2_create(16, 16, 2.5, 12, su2.SU2_COLD)
    made.append(h)
    su2.su2_set_sampler(h, su2.SU2_SAMPLER_KP)
    su2.su2_set_overrelax(h, 2)
    su2.su2_heatbath_sweep(h, 100)
    ws = []
    for _ in range(40):
        su2.su2_heatbath_sweep(h, 2)
        ws.append(su2.su2_wilson_loops(h, 4, 4))
    v = effective_potential(np.mean(ws, axis=0))[:, 1]  # T = 2 -> 3
    assert np.all(np.isfinite(v)) and np.all(np.diff(v) > 0), v
