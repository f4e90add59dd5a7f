"""Seeded synthetic workloads (shapes, couplings, seeds) used by the tests and
the benchmark.  Only input generation lives here -- none of the method's
arithmetic; the random numbers of the heat bath itself come from the Philox
counters on each side.

The shapes follow the paper: beta = 6.0 with a hot start (Sec. 4.1), 48^4 at
beta = 6.0 (abstract), cold starts on 8^4 (Fig. 4), Polyakov loops at finite
temporal extent (Sec. 4.2).
"""
from __future__ import annotations

import numpy as np

# (Ns, Nt, beta, start, seed): start 0 = cold, 1 = hot
PARITY_8 = dict(ns=8, nt=8, beta=2.3, start=1, seed=1, sweeps=10)
SCALE_24 = dict(ns=24, nt=24, beta=2.5, start=0, seed=2, therm=200, meas=1000, reunit_every=10)
PAPER_48 = dict(ns=48, nt=48, beta=6.0, start=1, seed=3)
FINITE_T = dict(ns=32, nt=4, betas=tuple(round(2.20 + 0.05 * i, 2) for i in range(9)), start=0, seed0=100)

BATCH_SHAPES = ((8, 8), (12, 4), (16, 6), (16, 16), (24, 8))


def batched(n: int = 64, seed: int = 5):
    """n lattices cycling through five shapes (8^4, 12^3x4, 16^3x6, 16^4,
    24^3x8), beta uniform in [1.5, 3.0] from a seeded numpy generator,
    Philox seeds 1000 + i, cold start."""
    rng = np.random.default_rng(seed)
    ns = [BATCH_SHAPES[i % 5][0] for i in range(n)]
    nt = [BATCH_SHAPES[i % 5][1] for i in range(n)]
    beta = [float(b) for b in 1.5 + 1.5 * rng.random(n)]
    seeds = [1000 + i for i in range(n)]
    return dict(ns=ns, nt=nt, beta=beta, seed=seeds, start=0)
