"""Training of the learned proposal on the GPU (tcgen05 BF16 contractions,
FP32 spline likelihood) against the binary64 oracle gradient, and the effect
of training on the proposal's acceptance."""
import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import learn, su2

pytestmark = pytest.mark.gpu


def oracle_pairs(ns, nt, beta, seed, sweeps, mu, parity, stride):
    links = oracle.hot_start(ns, nt, seed)
    for s in range(sweeps):
        oracle.heatbath_sweep(ns, nt, beta, seed, s, links, nthreads=8)
    return oracle.collect_pairs(ns, nt, beta, seed, sweeps, mu, parity, stride, links)


def bf16(x):
    """Round-to-nearest-even to BF16, returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_model_gradient(w, pairs):
    """The training step's data flow with BF16 operands for the four
    tensor-core contractions (as on the GPU) and the oracle's binary64 spline
    likelihood gradient in between."""
    W1, b1 = w[0:32].astype(float), w[32:64].astype(float)
    W2, b2 = w[64:1088].reshape(32, 32).astype(float), w[1088:1120].astype(float)
    W3, b3 = w[1120:1920].reshape(25, 32).astype(float), w[1920:1945].astype(float)
    g = np.zeros(1945)
    total = 0.0
    for bk, a in pairs.astype(float):
        s = (bk - w[1945]) * w[1946]
        h1 = np.maximum(W1 * s + b1, 0)
        h2 = np.maximum(bf16(W2) @ bf16(h1) + b2, 0)
        o = bf16(W3) @ bf16(h2) + b3
        l, go = oracle.nll_outputs(o, a)
        total += l
        dz2 = (bf16(W3).T @ bf16(go)) * (h2 > 0)
        dz1 = (bf16(W2).T @ bf16(dz2)) * (h1 > 0)
        g[0:32] += dz1 * s
        g[32:64] += dz1
        g[64:1088] += np.outer(dz2, h1).ravel()
        g[1088:1120] += dz2
        g[1120:1920] += np.outer(go, h2).ravel()
        g[1920:1945] += go
    return total / len(pairs), g / len(pairs)


def gpu_gradient(w, pairs):
    torch = pytest.importorskip("torch")
    dev = torch.from_numpy(np.ascontiguousarray(pairs)).cuda()
    tr = su2.su2_trainer_create(w, 1)
    try:
        return su2.su2_trainer_gradient(tr, dev.data_ptr(), pairs.shape[0])
    finally:
        su2.su2_trainer_destroy(tr)


def cosine(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.fixture(scope="module")
def pairs():
    return np.concatenate([oracle_pairs(8, 8, 2.4, 3, 3, 0, 0, 2), oracle_pairs(8, 8, 3.5, 4, 3, 1, 1, 2)])[:1024]


def weights_for(pairs, last_scale, seed=7):
    rng = np.random.default_rng(seed)
    w = learn.initial_weights(seed)
    w[1120:1920] = rng.normal(size=800) * last_scale
    w[1920:1945] = rng.normal(size=25) * last_scale
    w[1945] = float(pairs[:, 0].mean())
    w[1946] = float(1.0 / pairs[:, 0].std())
    return w


def test_gradient_matches_the_binary64_oracle(pairs):
    """Smooth spline (moderate outputs): BF16 contractions stay within 2%."""
    w = weights_for(pairs, 0.03)
    loss, g = gpu_gradient(w, pairs)
    want_loss, want = oracle.nll_grad(w.astype(np.float64), pairs)
    assert abs(loss - want_loss) < 1e-3 * max(1.0, abs(want_loss)), (loss, want_loss)
    assert cosine(g, want) > 0.999
    big = np.abs(want) > 0.05 * np.abs(want).max()
    rel = np.abs(g[big] - want[big]) / np.abs(want[big])
    assert rel.max() < 2e-2, (np.median(rel), rel.max())


def test_gradient_matches_the_bf16_model_where_the_likelihood_is_steep(pairs):
    """Large random outputs make bins whose knot derivatives are tiny; there
    the likelihood is so steep that BF16 operands move the gradient a lot.
    The GPU must still equal the same computation done with BF16 operands."""
    w = weights_for(pairs, 0.3)
    loss, g = gpu_gradient(w, pairs)
    want_loss, want = bf16_model_gradient(w, pairs)
    assert abs(loss - want_loss) < 1e-3 * max(1.0, abs(want_loss))
    assert cosine(g, want) > 0.999, cosine(g, want)


def test_training_lowers_the_loss_and_lifts_acceptance():
    torch = pytest.importorskip("torch")
    ns, nt, beta, seed = 12, 12, 3.0, 21
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT)
    try:
        su2.su2_heatbath_sweep(h, 30)
        pairs = learn.collect(h, ns, nt, 200_000)
        w, losses, s_lo, s_hi = learn.train(pairs, steps=600, batch=4096, lr=3e-3)
        assert np.all(np.isfinite(losses))
        assert losses[-50:].mean() < losses[:10].mean() - 0.1, (losses[:10].mean(), losses[-50:].mean())
        # untrained (near-uniform spline) against trained proposal on the lattice
        w0 = learn.initial_weights(0, float(w[1945]), float(w[1946]))
        su2.su2_set_proposal(h, w0, s_lo, s_hi, 256)
        _, _, st0 = su2.su2_learned_generate(h, 4, 0, 0.0)
        su2.su2_set_proposal(h, w, s_lo, s_hi, 256)
        _, _, st1 = su2.su2_learned_generate(h, 4, 0, 0.0)
        links = 4 * 4 * ns ** 3 * nt
        acc0, acc1 = sum(st0["accepted"]) / links, sum(st1["accepted"]) / links
        assert acc1 > 0.7 and acc1 > acc0 + 0.1, (acc0, acc1)
    finally:
        su2.su2_destroy(h)


def test_learned_chain_reproduces_the_plain_plaquette():
    """Exactness of the learned chain: same <P> as the plain heat bath within
    the combined statistical error (Gamma-method errors), 8^4 at beta = 2.3."""
    pytest.importorskip("torch")
    from paper_1010_1486_gb300.analysis import tau_int

    ns = nt = 8
    h = su2.su2_create(ns, nt, 2.3, 31, su2.SU2_HOT)
    try:
        su2.su2_heatbath_sweep(h, 100)
        pairs = learn.collect(h, ns, nt, 100_000)
        w, _, s_lo, s_hi = learn.train(pairs, steps=400, batch=4096, lr=3e-3)
        plain, _, _ = su2.su2_generate(h, 4000, 1, 0)
        su2.su2_set_proposal(h, w, s_lo, s_hi, 256)
        lp, _, st = su2.su2_learned_generate(h, 4000, 1, 0.7)
    finally:
        su2.su2_destroy(h)
    _, _, _, e_plain = tau_int(plain)
    t_l, _, _, e_learn = tau_int(lp)
    diff = lp.mean() - plain.mean()
    assert abs(diff) < 4 * np.hypot(e_plain, e_learn), (plain.mean(), lp.mean(), e_plain, e_learn)
    assert sum(st["accepted"]) / (st["learned_sweeps"] * 4 * ns ** 4) > 0.7
