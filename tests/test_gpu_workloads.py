"""The remaining workload shapes on the GPU:

- 24^4, beta = 2.5, cold start, reunitarisation every 10 sweeps: link for link
  with the oracle over 20 sweeps, then 200 + 1000 sweeps on the GPU with the
  plaquette every sweep and |a| = 1 to 1e-6 after every reunitarisation;
- the finite-temperature scan: 32^3 x 4 at beta = 2.20 ... 2.60 as one batch,
  link for link with the oracle over 3 sweeps;
- the paper's qualitative findings (Sec. 4.2): the plaquette rises with beta;
  the Polyakov loop |L| rises through the scan at Nt = 4;
- the binary32 error of the plaquette against the oracle's binary64 mode.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import su2, workloads

pytestmark = pytest.mark.gpu


def threads():
    return min(16, os.cpu_count() or 1)


def close(got, want, scale=0.05):
    return abs(got - want) <= 1e-6 * max(abs(want), scale)


def test_scale_24_cold_reunitarised_run():
    cfg = workloads.SCALE_24
    ns, nt, beta, seed = cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"]
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_COLD)
    try:
        plaq, poly, st = su2.su2_generate(h, 20, 1, cfg["reunit_every"])
        ref = oracle.cold_start(ns, nt)
        for s in range(20):
            oracle.heatbath_sweep(ns, nt, beta, seed, s, ref, nthreads=threads())
            if (s + 1) % 10 == 0:
                oracle.reunitarize(ns, nt, ref)
            assert close(plaq[s], oracle.plaquette(ns, nt, ref)) and close(poly[s], oracle.polyakov(ns, nt, ref)), s
        assert np.array_equal(su2.su2_get_links(h, ns, nt), ref)
        # the full run: thermalisation + measurement with reunitarisation every 10 sweeps
        therm, meas = cfg["therm"], cfg["meas"]
        su2.su2_generate(h, therm - 20, 0, 10)
        plaq, _, st = su2.su2_generate(h, meas, 1, 10)
        links = su2.su2_get_links(h, ns, nt)
        assert np.abs(np.linalg.norm(links.reshape(-1, 4).astype(np.float64), axis=1) - 1).max() <= 1e-6
        assert st["sampler_failures"] == 0
        # equilibrium SU(2) plaquette at beta = 2.5 is about 0.652; a wide check only
        assert 0.645 < plaq.mean() < 0.660, plaq.mean()
    finally:
        su2.su2_destroy(h)


def test_finite_temperature_scan_as_one_batch():
    cfg = workloads.FINITE_T
    betas = list(cfg["betas"])
    n = len(betas)
    ns, nt = [cfg["ns"]] * n, [cfg["nt"]] * n
    seeds = [cfg["seed0"] + i for i in range(n)]
    b = su2.su2_batch_create(ns, nt, betas, seeds, su2.SU2_COLD)
    try:
        plaq, poly, _ = su2.su2_batch_generate(b, n, 3, 1)
        for i in range(n):
            ref = oracle.cold_start(cfg["ns"], cfg["nt"])
            for s in range(3):
                oracle.heatbath_sweep(cfg["ns"], cfg["nt"], betas[i], seeds[i], s, ref, nthreads=threads())
            assert np.array_equal(su2.su2_batch_get_links(b, i, cfg["ns"], cfg["nt"]), ref), i
            assert close(plaq[2, i], oracle.plaquette(cfg["ns"], cfg["nt"], ref))
            assert close(poly[2, i], oracle.polyakov(cfg["ns"], cfg["nt"], ref))
    finally:
        su2.su2_batch_destroy(b)


def test_plaquette_and_polyakov_loop_rise_with_beta():
    """Sec. 4.2: <P> grows with beta; at Nt = 4, <|L|> grows through the
    deconfinement region (the scan 2.2 ... 2.6 brackets the transition)."""
    betas = [2.0, 2.2, 2.4, 2.6, 2.8]
    n = len(betas)
    b = su2.su2_batch_create([12] * n, [4] * n, betas, [500 + i for i in range(n)], su2.SU2_COLD)
    try:
        su2.su2_batch_sweep(b, 300)
        plaq, poly, _ = su2.su2_batch_generate(b, n, 1500, 1)
    finally:
        su2.su2_batch_destroy(b)
    p = plaq.mean(axis=0)
    l_abs = np.abs(poly).mean(axis=0)
    assert np.all(np.diff(p) > 0), p
    assert l_abs[-1] > 2 * l_abs[0] and l_abs[-1] > 0.2, l_abs


def test_binary32_plaquette_error_against_binary64():
    """The stated float error of the observables: per-site binary32 products
    and a binary64 sum against all-binary64 arithmetic on the same links."""
    ns = nt = 8
    h = su2.su2_create(ns, nt, 2.3, 1, su2.SU2_HOT)
    try:
        errs_p, errs_l = [], []
        for _ in range(10):
            su2.su2_heatbath_sweep(h, 1)
            links = su2.su2_get_links(h, ns, nt)
            errs_p.append(abs(su2.su2_plaquette(h) - oracle.plaquette_f64(ns, nt, links)))
            errs_l.append(abs(su2.su2_polyakov(h) - oracle.polyakov_f64(ns, nt, links)))
    finally:
        su2.su2_destroy(h)
    assert max(errs_p) < 2e-7 and max(errs_l) < 1e-6, (max(errs_p), max(errs_l))


def test_finite_temperature_scan_with_one_learned_proposal():
    """The 32^3 x 4 scan with the learned proposal and its plain fallback: one
    network trained on (beta k, a0) pairs pooled over the scan serves every
    beta; each lattice's learned chain keeps its acceptance above the
    fallback threshold and reproduces the plain chain's plaquette and |L|."""
    import torch

    from paper_1010_1486_gb300 import learn
    from paper_1010_1486_gb300.analysis import tau_int

    ns, nt = 32, 4
    betas = [2.2, 2.4, 2.6]
    lats = [su2.su2_create(ns, nt, b, 100 + i, su2.SU2_COLD) for i, b in enumerate(betas)]
    try:
        for h in lats:
            su2.su2_heatbath_sweep(h, 300)
        pairs = torch.cat([learn.collect(h, ns, nt, 100_000) for h in lats])
        w, losses, s_lo, s_hi = learn.train(pairs, steps=1500, batch=8192, lr=3e-3, seed=4, tail_steps=1500,
                                            tail_lr=3e-4)
        assert losses[-100:].mean() < losses[:100].mean()
        n = 1200
        for b, h in zip(betas, lats):
            su2.su2_set_proposal(h, w, s_lo, s_hi, 256)
            pl, ll, st = su2.su2_learned_generate(h, n, 1, 0.7)
            acc = sum(st["accepted"]) / (st["learned_sweeps"] * 4 * ns ** 3 * nt)
            assert st["learned_sweeps"] == n and acc > 0.85, (b, acc, st["plain_sweeps"])
            pp, lp, _ = su2.su2_generate(h, n, 1, 0)
            for lr_, pr_ in ((pl, pp), (np.abs(ll), np.abs(lp))):
                e = np.hypot(tau_int(lr_)[3], tau_int(pr_)[3])
                assert abs(lr_.mean() - pr_.mean()) < 5 * e, (b, lr_.mean(), pr_.mean(), e)
    finally:
        for h in lats:
            su2.su2_destroy(h)
