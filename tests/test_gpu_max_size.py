"""The largest lattice the library accepts: 64^3 x 2046, 4V = 2,145,386,496
links (34.3 GB), just below the 2^31-link limit that keeps every link index
in 32 bits (64^3 x 2048, exactly 2^31 links, is rejected: tests/test_abi.py).

Too large for the oracle to follow link by link, so the checks are the
properties that hold at any size:
- cold start: plaquette and Polyakov loop exactly 1;
- hot start (Haar links): |P| < 5 sigma with sigma = 1/(2 sqrt(6V)), and
  |L| < 5 sigma with sigma = 1/(2 sqrt(Ns^3)) (the half-trace of a Haar
  element has variance 1/4);
- one heat-bath sweep (Kennedy-Pendleton): every link finite and of unit
  norm to 1e-6, at least one trial per link update, the plaquette in (0, 1);
- reunitarization keeps every link of unit norm.
"""
import math

import pytest

from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu

NS, NT = 64, 2046
VOL = NS ** 3 * NT


def test_the_limit_is_where_the_library_puts_it():
    assert 4 * VOL < 2 ** 31 <= 4 * NS ** 3 * (NT + 2)


def test_cold_start_at_the_largest_size():
    lat = su2.su2_create(NS, NT, 2.3, 1, su2.SU2_COLD)
    try:
        assert su2.su2_plaquette(lat) == 1.0
        assert su2.su2_polyakov(lat) == 1.0
    finally:
        su2.su2_destroy(lat)


def test_hot_start_and_one_sweep_at_the_largest_size():
    lat = su2.su2_create(NS, NT, 2.3, 5, su2.SU2_HOT)
    try:
        assert su2.su2_check_links(lat, 1e-6) == (0, 0)
        p0 = su2.su2_plaquette(lat)
        l0 = su2.su2_polyakov(lat)
        assert abs(p0) < 5.0 / (2.0 * math.sqrt(6.0 * VOL)), p0
        assert abs(l0) < 5.0 / (2.0 * math.sqrt(NS ** 3)), l0
        su2.su2_set_sampler(lat, su2.SU2_SAMPLER_KP)
        st = su2.su2_heatbath_sweep(lat, 1, stats=True)
        assert st["link_updates"] == 4 * VOL
        assert sum(st["trials"]) >= 4 * VOL
        assert su2.su2_check_links(lat, 1e-6) == (0, 0)
        p1 = su2.su2_plaquette(lat)
        assert 0.0 < p1 < 1.0, p1
        assert math.isfinite(su2.su2_polyakov(lat))
        su2.su2_reunitarize(lat)
        assert su2.su2_check_links(lat, 1e-6) == (0, 0)
    finally:
        su2.su2_destroy(lat)
