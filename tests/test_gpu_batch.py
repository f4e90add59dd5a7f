"""Batched persistent sweep (many independent lattices in one cooperative
launch per sweep) against the CPU oracle run lattice by lattice."""
import os

import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import su2, workloads

pytestmark = pytest.mark.gpu

OBS_REL = 1e-6


def close(got, want, scale=0.05):
    return abs(got - want) <= OBS_REL * max(abs(want), scale)


def threads():
    return min(16, os.cpu_count() or 1)


def oracle_chains(cfg, sweeps):
    """Per lattice: links after each sweep, trial counts, P and L per sweep."""
    out = []
    for ns, nt, beta, seed in zip(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"]):
        links = oracle.hot_start(ns, nt, seed) if cfg["start"] == 1 else oracle.cold_start(ns, nt)
        trials = np.zeros(8, dtype=np.int64)
        plaq, poly = [], []
        for s in range(sweeps):
            trials += oracle.heatbath_sweep(ns, nt, beta, seed, s, links, nthreads=threads())
            plaq.append(oracle.plaquette(ns, nt, links))
            poly.append(oracle.polyakov(ns, nt, links))
        out.append(dict(links=links, trials=trials, plaq=plaq, poly=poly))
    return out


SMALL = dict(ns=[4, 6, 8, 4, 2, 10], nt=[4, 4, 8, 6, 2, 2], beta=[2.3, 1.7, 2.5, 0.0, 3.0, 2.1],
             seed=[11, 12, 13, 14, 15, 2 ** 40 + 16], start=1)


@pytest.mark.parametrize("use_stream", [False, True])
def test_batch_matches_oracle_lattice_by_lattice(use_stream):
    torch = pytest.importorskip("torch")
    cfg = SMALL
    sweeps = 3
    stream = torch.cuda.Stream() if use_stream else None
    b = su2.su2_batch_create(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"], cfg["start"], stream=stream)
    try:
        n = len(cfg["ns"])
        plaq, poly, st = su2.su2_batch_generate(b, n, sweeps, 1)
        ref = oracle_chains(cfg, sweeps)
        for i, r in enumerate(ref):
            got = su2.su2_batch_get_links(b, i, cfg["ns"][i], cfg["nt"][i])
            assert np.array_equal(got, r["links"]), i
            for s in range(sweeps):
                assert close(plaq[s, i], r["plaq"][s]), (i, s)
                assert close(poly[s, i], r["poly"][s]), (i, s)
        assert st["trials"] == [int(x) for x in sum(r["trials"] for r in ref)]
        assert st["sampler_failures"] == 0
        info = su2.su2_batch_info(b)
        assert info["sweep"] == sweeps and info["graphs"] == use_stream
        p_now = su2.su2_batch_plaquette(b, n)
        l_now = su2.su2_batch_polyakov(b, n)
        assert all(close(p_now[i], ref[i]["plaq"][-1]) for i in range(n))
        assert all(close(l_now[i], ref[i]["poly"][-1]) for i in range(n))
    finally:
        su2.su2_batch_destroy(b)


def test_every_queue_depth_gives_the_same_chain():
    cfg = SMALL
    results = []
    for depth in (1, 2, 4, 8):
        b = su2.su2_batch_create(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"], cfg["start"])
        try:
            su2.su2_batch_set_config(b, depth, 0 if depth != 4 else 37)
            su2.su2_batch_sweep(b, 2)
            results.append([su2.su2_batch_get_links(b, i, cfg["ns"][i], cfg["nt"][i]) for i in range(len(cfg["ns"]))])
        finally:
            su2.su2_batch_destroy(b)
    for other in results[1:]:
        assert all(np.array_equal(x, y) for x, y in zip(results[0], other))


def test_autotune_keeps_the_chain():
    torch = pytest.importorskip("torch")
    cfg = SMALL
    stream = torch.cuda.Stream()
    b = su2.su2_batch_create(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"], cfg["start"], stream=stream)
    try:
        su2.su2_batch_sweep(b, 1)
        depth, grid = su2.su2_batch_autotune(b, 2)
        assert depth in (1, 2, 4, 8) and grid > 0
        assert su2.su2_batch_info(b)["sweep"] == 1
        su2.su2_batch_sweep(b, 2)
        ref = oracle_chains(cfg, 3)
        for i, r in enumerate(ref):
            assert np.array_equal(su2.su2_batch_get_links(b, i, cfg["ns"][i], cfg["nt"][i]), r["links"])
    finally:
        su2.su2_batch_destroy(b)


def test_sixty_four_uneven_lattices():
    """64 lattices of 8^4, 12^3x4, 16^3x6, 16^4, 24^3x8, beta in [1.5, 3],
    seeds 1000+i, cold start: two sweeps with measurements, every lattice
    compared link for link."""
    torch = pytest.importorskip("torch")
    cfg = workloads.batched()
    n = len(cfg["ns"])
    b = su2.su2_batch_create(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"], cfg["start"],
                             stream=torch.cuda.Stream())
    try:
        plaq, poly, st = su2.su2_batch_generate(b, n, 2, 1)
        ref = oracle_chains(cfg, 2)
        for i, r in enumerate(ref):
            assert np.array_equal(su2.su2_batch_get_links(b, i, cfg["ns"][i], cfg["nt"][i]), r["links"]), i
            assert close(plaq[1, i], r["plaq"][1]) and close(poly[1, i], r["poly"][1]), i
        assert st["trials"] == [int(x) for x in sum(r["trials"] for r in ref)]
    finally:
        su2.su2_batch_destroy(b)


def test_grid_barrier_wait_gives_up_and_reports():
    # nothing completes the barrier: every block must stop after ~2 ms
    assert su2.su2_selftest_barrier_timeout(8, 2_000_000) == 8
    # the context stays usable afterwards
    h = su2.su2_create(4, 4, 2.3, 1, su2.SU2_COLD)
    try:
        assert su2.su2_plaquette(h) == 1.0
    finally:
        su2.su2_destroy(h)


def test_batch_rejects_bad_arguments():
    with pytest.raises(su2.SU2Error):
        su2.su2_batch_create([4, 5], [4, 4], [2.0, 2.0], [1, 2])
    with pytest.raises(su2.SU2Error):
        su2.su2_batch_create([4], [4], [float("nan")], [1])


def oracle_chains_kp(cfg, sweeps):
    out = []
    for ns, nt, beta, seed in zip(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"]):
        links = oracle.hot_start(ns, nt, seed) if cfg["start"] == 1 else oracle.cold_start(ns, nt)
        trials = np.zeros(8, dtype=np.int64)
        plaq = []
        for s in range(sweeps):
            trials += oracle.heatbath_sweep_kp(ns, nt, beta, seed, s, links, nthreads=threads())
            plaq.append(oracle.plaquette(ns, nt, links))
        out.append(dict(links=links, trials=trials, plaq=plaq))
    return out


@pytest.mark.parametrize("depth,block", [(4, 128), (2, 256), (8, 64), (1, 128)])
def test_kennedy_pendleton_batch_matches_the_oracle(depth, block):
    """The batch with the Kennedy-Pendleton sampler: every lattice bitwise the
    oracle's KP chain (beta k < 2 links by Creutz's method included: beta 0
    and 0.5 lattices), trial counts equal, fused plaquettes within 1e-6."""
    cfg = dict(SMALL)
    cfg["beta"] = [2.3, 1.7, 6.0, 0.0, 3.0, 0.5]
    sweeps = 3
    b = su2.su2_batch_create(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"], cfg["start"])
    try:
        su2.su2_batch_set_sampler(b, su2.SU2_SAMPLER_KP)
        su2.su2_batch_set_launch(b, depth, block, 0)
        assert su2.su2_batch_launch_info(b)[:2] == (depth, block)
        n = len(cfg["ns"])
        plaq, _, st = su2.su2_batch_generate(b, n, sweeps, 1)
        ref = oracle_chains_kp(cfg, sweeps)
        for i, r in enumerate(ref):
            assert np.array_equal(su2.su2_batch_get_links(b, i, cfg["ns"][i], cfg["nt"][i]), r["links"]), i
            for s in range(sweeps):
                assert close(plaq[s, i], r["plaq"][s]), (i, s)
        assert st["trials"] == [int(x) for x in sum(r["trials"] for r in ref)]
        assert st["sampler_failures"] == 0
    finally:
        su2.su2_batch_destroy(b)


def test_kennedy_pendleton_batch_of_64_uneven_lattices():
    cfg = workloads.batched(64, seed=5)
    sweeps = 2
    b = su2.su2_batch_create(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"], cfg["start"])
    try:
        su2.su2_batch_set_sampler(b, su2.SU2_SAMPLER_KP)
        su2.su2_batch_autotune(b, 2)
        su2.su2_batch_sweep(b, sweeps)
        for i in range(0, 64, 7):
            links = oracle.cold_start(cfg["ns"][i], cfg["nt"][i])
            for s in range(sweeps):
                oracle.heatbath_sweep_kp(cfg["ns"][i], cfg["nt"][i], cfg["beta"][i], cfg["seed"][i], s, links,
                                         nthreads=threads())
            assert np.array_equal(su2.su2_batch_get_links(b, i, cfg["ns"][i], cfg["nt"][i]), links), i
    finally:
        su2.su2_batch_destroy(b)
