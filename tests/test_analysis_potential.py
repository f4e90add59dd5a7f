"""Host helpers for the static potential: effective masses of synthetic
Wilson loops W = C(R) exp(-V(R) T) and the Cornell fit recover V and its
parameters exactly."""
import numpy as np

from paper_1010_1486_gb300.analysis import cornell_fit, effective_potential


def test_effective_potential_and_cornell_fit():
    r = np.arange(1, 7, dtype=np.float64)
    v0, alpha, sigma = 0.6, 0.28, 0.05
    v = v0 - alpha / r + sigma * r
    t = np.arange(1, 9, dtype=np.float64)
    c = 0.9 - 0.05 * r
    w = c[:, None] * np.exp(-v[:, None] * t[None, :])
    ve = effective_potential(w)
    assert ve.shape == (6, 7)
    assert np.allclose(ve, v[:, None], atol=1e-12)
    assert np.allclose(cornell_fit(r, v), (v0, alpha, sigma), atol=1e-10)


def test_effective_potential_marks_non_positive_ratios():
    w = np.array([[0.5, 0.25, -0.1], [0.4, 0.0, 0.1]])
    ve = effective_potential(w)
    assert abs(ve[0, 0] - np.log(2)) < 1e-15
    assert np.isnan(ve[0, 1]) and np.isnan(ve[1, 0]) and np.isnan(ve[1, 1])
