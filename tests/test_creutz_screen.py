"""The screened Creutz trial: a rejection or acceptance is decided from the
hardware base-2 logarithm unless the trial falls within a slack band of the
acceptance boundary, where the exact test runs.  Its verdict is the exact
test's only if two error bounds hold over every float x in [2^-34, 1] (the
range x = e + r1 (1 - e) takes, r1 >= 2^-33):

  log_series:  |L(x) - ln x| <= 1e-6 |ln x| + 1e-7
  __log2f:     |lg2(x) - log2 x| <= 2^-22 on [1/2, 1], <= 2.4e-7 |log2 x| below

The first is checked here on the CPU through the oracle's log (the same
binary32 function as the kernels' log_series, operation for operation), and on
the GPU as bitwise equality of the two over the same floats; the second on the
GPU.  A third test runs the screen against the exact test on trials placed at
the acceptance boundary.
"""
import numpy as np
import pytest

import oracle

LO_BITS = np.float32(2.0 ** -34).view(np.uint32)
ONE_BITS = np.float32(1.0).view(np.uint32)
CHUNK = 1 << 23


def every_float(lo=LO_BITS, hi=ONE_BITS):
    """All binary32 values in [2^-34, 1], in chunks of 2^23."""
    for b0 in range(int(lo), int(hi) + 1, CHUNK):
        bits = np.arange(b0, min(b0 + CHUNK, int(hi) + 1), dtype=np.uint32)
        yield bits.view(np.float32)


def test_log_series_error_bound_every_float():
    worst = 0.0
    for x in every_float():
        got = oracle.logf(x).astype(np.float64)
        want = np.log(x.astype(np.float64))
        err = np.abs(got - want) - (1e-6 * np.abs(want) + 1e-7)
        worst = max(worst, float(err.max()))
    assert worst <= 0.0, worst


def random_trials(rng, n, near_boundary):
    """(r1, r2, 1/(beta k), exp(-2 beta k)) rows over beta k in [0.05, 60];
    near_boundary puts r2 within a relative 2e-4 of sqrt(1 - a0^2)."""
    bk = np.exp(rng.uniform(np.log(0.05), np.log(60.0), n))
    ibk = (1.0 / bk).astype(np.float32)
    e = np.where(bk <= 21.0, np.exp(-2.0 * bk), 0.0).astype(np.float32)
    # r1 as the kernels draw it for a logarithm: w 2^-32 + 2^-33
    w = rng.integers(0, 1 << 32, n, dtype=np.uint64)
    r1 = (w.astype(np.float32).astype(np.float64) * 2.0 ** -32 + 2.0 ** -33).astype(np.float32)
    if near_boundary:
        x = r1.astype(np.float64) * (1.0 - e) + e
        t = -np.log(x) / bk
        R = np.clip(t * (2.0 - t), 0.0, 1.0)
        r2 = np.sqrt(R) * (1.0 + rng.uniform(-2e-4, 2e-4, n))
        r2 = np.clip(r2, 2.0 ** -24, 1.0).astype(np.float32)
    else:
        r2 = ((rng.integers(0, 1 << 24, n) + 1) * 2.0 ** -24).astype(np.float32)
    return np.stack([r1, r2, ibk, e], axis=1).astype(np.float32)


@pytest.mark.gpu
def test_gpu_log_series_every_float_matches_oracle():
    from paper_1010_1486_gb300 import su2

    for x in every_float():
        got = su2.su2_selftest_math(0, x)
        assert np.array_equal(got.view(np.uint32), oracle.logf(x).view(np.uint32))


@pytest.mark.gpu
def test_gpu_hardware_log2_error_bound_every_float():
    from paper_1010_1486_gb300 import su2

    for x in every_float():
        got = su2.su2_selftest_math(3, x).astype(np.float64)
        want = np.log2(x.astype(np.float64))
        bound = np.where(x >= 0.5, 2.0 ** -22, 2.4e-7 * np.abs(want))
        assert np.all(np.abs(got - want) <= bound)


@pytest.mark.gpu
@pytest.mark.parametrize("near_boundary", [False, True])
def test_gpu_screen_agrees_with_exact_test(near_boundary):
    from paper_1010_1486_gb300 import su2

    rng = np.random.default_rng(11 + near_boundary)
    q = random_trials(rng, 1 << 22, near_boundary)
    screen, exact = su2.su2_selftest_math(4, q)
    assert set(np.unique(screen)) <= {0.0, 1.0, 2.0}
    decided = screen != 2.0
    assert np.array_equal(screen[decided], exact[decided])
    undecided = float(np.mean(~decided))
    if near_boundary:
        # the band is a part of the +-2e-4 window around the boundary
        assert 0.0 < undecided < 0.5
    else:
        assert undecided < 1e-3
    # the Haar branch (1/(beta k) = 0) always goes to the exact test
    h = q[:1024].copy()
    h[:, 2] = 0.0
    h[:, 3] = 0.0
    hs, _ = su2.su2_selftest_math(4, h)
    assert np.all(hs == 2.0)
