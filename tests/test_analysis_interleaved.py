"""analysis.interleaved_offset: the offset of one Monte Carlo form against
a reference form from interleaved blocks, with the reference interpolated at
each block's position so that a slow drift of the chain cancels."""
import numpy as np
import pytest

from paper_1010_1486_gb300.analysis import interleaved_offset


def test_linear_drift_cancels_only_with_the_interpolated_reference():
    n, drift, true_offset = 40, 2.4e-7, 1.5e-7
    rng = np.random.default_rng(3)
    ref = 0.87 + drift * np.arange(n + 1) + rng.normal(0.0, 1e-9, n + 1)
    for f in (0.2, 1.0 / 3.0, 2.0 / 3.0, 0.7):
        test = 0.87 + drift * (np.arange(n) + f) + true_offset + rng.normal(0.0, 1e-9, n)
        m, se = interleaved_offset(test, ref, f)
        assert abs(m - true_offset) < 5 * se + 1e-12
        # the midpoint reference is off by (f - 1/2) times the drift per round
        m_mid, _ = interleaved_offset(test, ref, 0.5)
        assert m_mid - true_offset == pytest.approx((f - 0.5) * drift, rel=0.05, abs=2e-9)


def test_error_is_the_spread_of_the_block_offsets():
    rng = np.random.default_rng(5)
    ref = rng.normal(0.0, 1.0, 101)
    test = rng.normal(0.0, 1.0, 100)
    m, se = interleaved_offset(test, ref, 0.25)
    d = test - (ref[:-1] + 0.25 * (ref[1:] - ref[:-1]))
    assert m == pytest.approx(d.mean()) and se == pytest.approx(d.std(ddof=1) / 10.0)


def test_block_counts_are_checked():
    with pytest.raises(ValueError):
        interleaved_offset([1.0, 2.0], [1.0, 2.0], 0.5)
    with pytest.raises(ValueError):
        interleaved_offset([1.0], [1.0, 2.0], 0.5)


def test_block_drift_recovers_a_linear_trend():
    from paper_1010_1486_gb300.analysis import block_drift

    rng = np.random.default_rng(3)
    k = np.arange(40)
    b = 0.5 + 2e-3 * k + rng.normal(0, 1e-3, 40)
    slope, err, block_err = block_drift(b)
    assert abs(slope - 2e-3) < 4 * err
    assert 0.6e-3 < block_err < 1.4e-3
    flat = block_drift(0.5 + rng.normal(0, 1e-3, 40))
    assert abs(flat[0]) < 4 * flat[1]
