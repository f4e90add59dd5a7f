"""Failure detection without a GPU fault: the sampler's trial cap (forced low
with su2_set_trial_cap), the link-health check (su2_check_links) and the
bounded mbarrier wait of the learned phase's table copy (made to run out on
a barrier that nothing completes).  A link
whose draw reaches the cap keeps its old value and the status is
SU2_E_SAMPLER; every other link equals the oracle's uncapped draw bit for bit
(the draws are the same counters).  Non-finite links give SU2_E_NUMERIC."""
import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu

SU2_E_SAMPLER, SU2_E_NUMERIC = 4, 6


def parity_sites(ns, nt, parity):
    s = np.arange(ns ** 3 * nt)
    x, y, z, t = s % ns, (s // ns) % ns, (s // ns ** 2) % ns, s // ns ** 3
    return s[(x + y + z + t) % 2 == parity]


@pytest.mark.parametrize("sampler,ns,cap", [(su2.SU2_SAMPLER_CREUTZ, 8, 2), (su2.SU2_SAMPLER_CREUTZ, 8, 4),
                                            (su2.SU2_SAMPLER_KP, 24, 2)])
def test_trial_cap_keeps_the_old_link_and_reports(sampler, ns, cap):
    nt, beta, seed, mu, parity = ns, 6.0, 7, 0, 0
    # cold start: beta k = 36 everywhere; Creutz accepts 0.23 of trials, KP
    # about 0.99 (so KP needs 24^4 for a few dozen links beyond two trials)
    want = oracle.cold_start(ns, nt)
    old = want.copy()
    if sampler == su2.SU2_SAMPLER_KP:
        oracle.heatbath_phase_kp(ns, nt, beta, seed, 0, mu, parity, want, nthreads=8)
    else:
        oracle.heatbath_phase(ns, nt, beta, seed, 0, mu, parity, want)
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_COLD)
    try:
        su2.su2_set_sampler(h, sampler)
        su2.su2_set_trial_cap(h, cap)
        su2.su2_heatbath_phase(h, mu, parity)
        with pytest.raises(su2.SU2Error) as err:
            su2.su2_sync(h)
        assert err.value.status == SU2_E_SAMPLER
        got = su2.su2_get_links(h, ns, nt)
        sites = parity_sites(ns, nt, parity)
        g, w, o = got[sites, mu], want[sites, mu], old[sites, mu]
        same_as_oracle = np.all(g.view(np.uint32) == w.view(np.uint32), axis=1)
        kept = np.all(g.view(np.uint32) == o.view(np.uint32), axis=1)
        assert np.all(same_as_oracle | kept)
        assert kept.sum() > 0 and same_as_oracle.sum() > 0
        # the other links are untouched
        others = np.ones(got.shape[:2], dtype=bool)
        others[sites, mu] = False
        assert np.array_equal(got[others].view(np.uint32), old[others].view(np.uint32))
        # the flag was cleared by su2_sync; with the default cap the next sweep is clean
        su2.su2_set_trial_cap(h, 4096)
        su2.su2_heatbath_sweep(h, 1, stats=True)
        su2.su2_sync(h)
    finally:
        su2.su2_destroy(h)


def test_trial_cap_change_recaptures_the_generation_graph():
    """On a lattice with a stream su2_generate replays a captured graph; the
    cap is part of its signature, so lowering it must take effect at once."""
    import torch

    h = su2.su2_create(8, 8, 6.0, 7, su2.SU2_COLD, stream=torch.cuda.Stream())
    try:
        su2.su2_generate(h, 2, 1, 0)  # captured and replayed at the default cap
        su2.su2_set_trial_cap(h, 2)
        with pytest.raises(su2.SU2Error) as err:
            su2.su2_generate(h, 1, 1, 0)
        assert err.value.status == SU2_E_SAMPLER
        su2.su2_set_trial_cap(h, 4096)
        su2.su2_generate(h, 2, 1, 0)
    finally:
        su2.su2_destroy(h)


def test_trial_cap_arguments():
    h = su2.su2_create(4, 4, 2.0, 1, su2.SU2_COLD)
    try:
        for bad in (0, 1, 3, 4097, 5000):
            with pytest.raises(su2.SU2Error):
                su2.su2_set_trial_cap(h, bad)
        su2.su2_set_trial_cap(h, 4096)
    finally:
        su2.su2_destroy(h)


def test_check_links_counts_bad_links():
    ns, nt = 6, 4
    h = su2.su2_create(ns, nt, 2.3, 3, su2.SU2_HOT)
    try:
        su2.su2_heatbath_sweep(h, 5)
        assert su2.su2_check_links(h, 1e-6) == (0, 0)
        links = su2.su2_get_links(h, ns, nt)
        links[5, 2] *= 1.001           # off the unit sphere
        su2.su2_set_links(h, links)
        assert su2.su2_check_links(h, 1e-6) == (0, 1)
        assert su2.su2_check_links(h, 1e-2) == (0, 0)
        links[7, 1, 3] = np.nan         # non-finite
        links[8, 0, 0] = np.inf
        su2.su2_set_links(h, links)
        with pytest.raises(su2.SU2Error) as err:
            su2.su2_check_links(h, 1e-6)
        assert err.value.status == SU2_E_NUMERIC
        su2.su2_reunitarize(h)  # NaN stays NaN; the scaled link is repaired
        with pytest.raises(su2.SU2Error):
            su2.su2_check_links(h, 1e-6)
        with pytest.raises(su2.SU2Error):
            su2.su2_check_links(h, -1.0)
    finally:
        su2.su2_destroy(h)


def test_mbarrier_wait_gives_up_and_reports():
    """Every block's wait on an mbarrier that nothing completes gives up
    after its polls, and the context stays usable."""
    assert su2.su2_selftest_mbar_timeout(8, 1000) == 8
    assert su2.su2_selftest_mbar_timeout(152, 1 << 16) == 152
    lat = su2.su2_create(4, 4, 2.3, 1, su2.SU2_COLD)
    try:
        assert su2.su2_plaquette(lat) == 1.0
    finally:
        su2.su2_destroy(lat)
