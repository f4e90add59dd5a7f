"""The Polyakov loop kernel on time extents that exercise its split of the
time direction: four lanes per spatial site, each multiplying a quarter of
the Nt links (in batches of twelve loads), the quarters combined in order.

Against the oracle's binary64 loop on the same links: per site the binary32
product of Nt quaternions carries at most about Nt x 6e-8 of relative
rounding, so the mean over sites stays within 1e-7 x Nt of the binary64
value.  Extents: quarters shorter than a batch, empty quarters (Nt = 2, 6),
and quarters of one, two and three batches (Nt = 50, 98, 146).
"""
import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ns,nt", [(4, 2), (2, 6), (4, 10), (2, 26), (4, 50), (2, 98), (2, 146)])
def test_polyakov_loop_on_split_time_extents(ns, nt):
    lat = su2.su2_create(ns, nt, 2.3, 7 + nt, su2.SU2_HOT)
    try:
        for sweeps in (0, 2):
            su2.su2_heatbath_sweep(lat, sweeps)
            links = su2.su2_get_links(lat, ns, nt)
            want = oracle.polyakov_f64(ns, nt, links)
            got = su2.su2_polyakov(lat)
            assert abs(got - want) <= 1e-7 * nt, (ns, nt, sweeps, got, want)
    finally:
        su2.su2_destroy(lat)


def test_polyakov_loop_of_a_uniform_field_is_a_closed_form():
    """Every link the same SU(2) element a = (cos th, sin th n): the loop at
    each site is a^Nt = cos(Nt th) + i sin(Nt th) n.sigma, so L = cos(Nt th),
    here for the binary32-rounded a: |a|^Nt cos(Nt th') with th' its angle."""
    ns, nt, th = 4, 22, 0.3
    n = np.array([0.48, 0.6, 0.64])
    n /= np.linalg.norm(n)
    a = np.concatenate([[np.cos(th)], np.sin(th) * n]).astype(np.float32)
    links = np.broadcast_to(a, (ns * ns * ns * nt, 4, 4)).copy()
    lat = su2.su2_create(ns, nt, 2.3, 1, su2.SU2_COLD)
    try:
        su2.su2_set_links(lat, links)
        got = su2.su2_polyakov(lat)
    finally:
        su2.su2_destroy(lat)
    a64 = a.astype(np.float64)
    r = np.linalg.norm(a64)
    want = r ** nt * np.cos(nt * np.arctan2(np.linalg.norm(a64[1:]), a64[0]))
    assert abs(want - np.cos(nt * th)) < 1e-5
    assert abs(got - want) <= 2e-6, (got, want)
