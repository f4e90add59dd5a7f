"""Writes learned_weights.txt: a proposal network trained on the CPU with the
oracle alone, for the tests that compare the proposal table with the network.

The learned proposal has no counterpart in the paper, which fixes only the
target law of a0 (Sec. 2): p(a0) ~ sqrt(1 - a0^2) exp(beta k a0).  The pairs
here are exact draws from that law (the oracle's Creutz sampler at fixed
beta k), with beta k spread log-uniformly over [1, 40]: the range that the
lattices of the tests and the 48^4, beta = 6 benchmark visit.  The network is
fitted by maximum likelihood with the oracle's binary64 gradient and Adam, so
that the tests see a trained proposal (a few kinks of its ReLU units inside
the range, sharp splines at large beta k), not random weights.  Nothing here
comes from the CUDA path.

Run from the repository root:  python tests/golden/make_learned_weights.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "learned_weights.txt")
BK_LO, BK_HI = 1.0, 40.0
N_BK, PER_BK = 400, 500
STAGES = ((1500, 3e-3), (500, 3e-4))
BATCH = 4096


def training_pairs():
    bks = np.exp(np.linspace(np.log(BK_LO), np.log(BK_HI), N_BK)).astype(np.float32)
    pairs = []
    for i, bk in enumerate(bks):
        a0, trials = oracle.creutz_a0_many(float(bk), 11, PER_BK, eo0=i * PER_BK)
        assert (trials > 0).all()
        pairs.append(np.stack([np.full(PER_BK, bk, np.float32), a0], axis=1))
    return np.concatenate(pairs).astype(np.float32)


def init_weights(rng, mean, scale):
    w = np.zeros(oracle.N_WEIGHTS)
    w[0:32] = rng.normal(size=32)                               # W1 (fan-in 1)
    w[32:64] = rng.uniform(-1.0, 1.0, 32)                       # b1: kinks spread over s
    w[64:1088] = rng.normal(size=1024) * np.sqrt(2.0 / 32.0)    # W2
    w[1120:1920] = rng.normal(size=800) * 0.01                  # W3: start near the uniform spline
    w[oracle.N_TRAIN] = mean
    w[oracle.N_TRAIN + 1] = scale
    return w


def train(pairs, seed=12):
    rng = np.random.default_rng(seed)
    bk = pairs[:, 0].astype(np.float64)
    w = init_weights(rng, float(np.float32(bk.mean())), float(np.float32(1.0 / bk.std())))
    m = np.zeros(oracle.N_TRAIN)
    v = np.zeros(oracle.N_TRAIN)
    t = 0
    for steps, lr in STAGES:
        for _ in range(steps):
            batch = pairs[rng.integers(0, pairs.shape[0], BATCH)]
            _, g = oracle.nll_grad(w, batch)
            t += 1
            m = 0.9 * m + 0.1 * g
            v = 0.999 * v + 0.001 * g * g
            mh = m / (1 - 0.9 ** t)
            vh = v / (1 - 0.999 ** t)
            w[:oracle.N_TRAIN] -= lr * mh / (np.sqrt(vh) + 1e-8)
    return w.astype(np.float32)


if __name__ == "__main__":
    pairs = training_pairs()
    w = train(pairs)
    nll, _ = oracle.nll_grad(w, pairs, want_grad=False)
    with open(OUT, "w") as f:
        f.write("# proposal network (1945 weights, then input mean and scale), binary32, written by\n")
        f.write(f"# make_learned_weights.py from oracle/ only; beta k in [{BK_LO}, {BK_HI}], "
                f"mean -log q on the training pairs {nll:.6f}\n")
        for x in w:
            f.write(f"{float(x)!r}\n")
    print(OUT, nll)
