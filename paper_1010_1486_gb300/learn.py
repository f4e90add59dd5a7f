"""Host side of the learned proposal: initial weights, and the pipeline
collect pairs on the lattice -> train on the GPU -> install the proposal.
Every computation runs in libsu2's kernels; this module only sequences calls.
"""
from __future__ import annotations

import numpy as np

from . import su2

N_WEIGHTS = su2.N_WEIGHTS


def initial_weights(seed: int = 0, mean: float = 0.0, scale: float = 1.0) -> np.ndarray:
    """He-style random initial weights (numpy generator), zero biases; the
    last layer starts small so the first spline is close to uniform."""
    rng = np.random.default_rng(seed)
    w = np.zeros(N_WEIGHTS, dtype=np.float32)
    w[0:32] = rng.normal(size=32) * np.sqrt(2.0)
    w[64:1088] = rng.normal(size=1024) * np.sqrt(2.0 / 32)
    w[1120:1920] = rng.normal(size=800) * 0.01
    w[1945], w[1946] = mean, scale
    return w


def collect(lat: int, ns: int, nt: int, n_pairs: int, sweeps_between: int = 1, stride: int = 0):
    """About n_pairs (beta k, a0) pairs collected on the lattice, cycling over
    the 8 phases with `sweeps_between` heat-bath sweeps between collections.
    Returns a float32 CUDA tensor of shape (n, 2)."""
    import torch

    vh = ns ** 3 * nt // 2
    if stride <= 0:
        stride = max(1, vh // max(1, n_pairs // 8))
    per = (vh + stride - 1) // stride
    rounds = max(1, (n_pairs + per - 1) // per)
    buf = torch.zeros((rounds * per, 2), dtype=torch.float32, device="cuda")
    for r in range(rounds):
        su2.su2_heatbath_sweep(lat, sweeps_between)
        mu, par = (r // 2) % 4, r % 2
        view = buf[r * per:(r + 1) * per]
        su2.su2_collect_pairs(lat, mu, par, stride, view.data_ptr(), per)
    torch.cuda.synchronize()
    return buf[:n_pairs] if buf.shape[0] > n_pairs else buf


def train(pairs, steps: int = 2000, batch: int = 4096, lr: float = 1e-3, seed: int = 0, tail_steps: int = 0,
          tail_lr: float | None = None):
    """Trains a proposal on device pairs; returns (weights, losses, s_lo, s_hi)
    where [s_lo, s_hi] is the range of normalised inputs seen in the data.
    `steps` Adam steps at `lr`, then `tail_steps` more at `tail_lr` (the
    optimizer state carries over)."""
    w0 = initial_weights(seed)
    tr = su2.su2_trainer_create(w0, seed)
    try:
        n = pairs.shape[0]
        su2.su2_trainer_set_input_scaling(tr, pairs.data_ptr(), n)
        losses = su2.su2_trainer_fit(tr, pairs.data_ptr(), n, steps, batch, lr)
        if tail_steps > 0:
            tail = su2.su2_trainer_fit(tr, pairs.data_ptr(), n, tail_steps, batch,
                                       tail_lr if tail_lr is not None else lr / 10)
            losses = np.concatenate([losses, tail])
        w = su2.su2_trainer_get_weights(tr)
    finally:
        su2.su2_trainer_destroy(tr)
    bk = pairs[:, 0]
    s_lo = float(((bk.min() - float(w[1945])) * float(w[1946])).item()) - 0.5
    s_hi = float(((bk.max() - float(w[1945])) * float(w[1946])).item()) + 0.5
    return w, losses, s_lo, s_hi
