"""The plaquette measured inside a sweep (odd phases of mu = 1, 2, 3 add
(1/2) Tr U'S over the staple terms of nu < mu) equals the separate plaquette
kernel on the same links, for every kind of sweep that can end a measured
step: Creutz, Kennedy-Pendleton, over-relaxation, learned and its plain
fallback; on ragged, self-wrapping and full-size lattices."""
import numpy as np
import pytest

from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu


def close(a, b):
    return abs(a - b) <= 2e-7 * max(abs(b), 0.05)


def fused_then_separate(h, sweeps, generate):
    for _ in range(sweeps):
        p_fused = generate()
        p_sep = su2.su2_plaquette(h)
        assert close(p_fused, p_sep), (p_fused, p_sep)
    return p_fused


@pytest.mark.parametrize("ns,nt,beta,sampler,n_or", [
    (8, 8, 2.3, su2.SU2_SAMPLER_CREUTZ, 0), (6, 4, 2.0, su2.SU2_SAMPLER_CREUTZ, 0),
    (2, 2, 2.3, su2.SU2_SAMPLER_CREUTZ, 0), (10, 2, 6.0, su2.SU2_SAMPLER_KP, 0),
    (8, 4, 6.0, su2.SU2_SAMPLER_KP, 0), (6, 6, 2.5, su2.SU2_SAMPLER_CREUTZ, 2),
    (4, 6, 6.0, su2.SU2_SAMPLER_KP, 1)])
def test_heat_bath_and_overrelaxation(ns, nt, beta, sampler, n_or):
    h = su2.su2_create(ns, nt, beta, 7, su2.SU2_HOT)
    try:
        su2.su2_set_sampler(h, sampler)
        su2.su2_set_overrelax(h, n_or)
        fused_then_separate(h, 4, lambda: su2.su2_generate(h, 1, 1, 0)[0][0])
    finally:
        su2.su2_destroy(h)


@pytest.mark.parametrize("scale,threshold", [(0.02, 0.0), (0.2, 0.999)])
def test_learned_and_its_fallback(scale, threshold):
    """A near-uniform proposal (learned sweeps only) and a poor one with a
    threshold no sweep reaches (learned and plain sweeps alternate)."""
    rng = np.random.default_rng(3)
    w = np.zeros(su2.N_WEIGHTS, dtype=np.float32)
    w[:1945] = rng.normal(size=1945) * scale
    w[1945], w[1946] = 7.0, 0.5
    h = su2.su2_create(6, 6, 2.3, 5, su2.SU2_HOT)
    try:
        su2.su2_set_proposal(h, w, -3.0, 3.0, 64)
        fused_then_separate(h, 4, lambda: su2.su2_learned_generate(h, 1, 1, threshold)[0][0])
    finally:
        su2.su2_destroy(h)


def test_full_size_48():
    h = su2.su2_create(48, 48, 6.0, 3, su2.SU2_HOT)
    try:
        su2.su2_heatbath_sweep(h, 2)
        p = fused_then_separate(h, 2, lambda: su2.su2_generate(h, 1, 1, 0)[0][0])
        assert 0.3 < p < 0.9
    finally:
        su2.su2_destroy(h)
