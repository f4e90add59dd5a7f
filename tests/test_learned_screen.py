"""The screened Metropolis test of the learned step: accept iff Delta >= 0 or
u1 <= exp(Delta), Delta = beta k (a' - a) + log(ratio), decided from hardware
base-2 logarithms unless the estimate falls within a slack band, where the
exact arithmetic runs.  Every decided verdict must be the exact one; the
inputs are typical (a' and a from the heat-bath law's range, spline slopes
over six decades) and placed at the two boundaries (Delta = 0, and
u1 = exp(Delta))."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def near_one(rng, bk, n):
    # a = 1 - g / (beta k), g ~ Gamma(3/2): the bulk of the heat-bath law
    return np.clip(1.0 - rng.gamma(1.5, 1.0, n) / bk, -0.999, 0.999999)


def octuples(rng, n, mode):
    bk = np.exp(rng.uniform(np.log(2.0), np.log(60.0), n))
    a_new = near_one(rng, bk, n)
    acur = near_one(rng, bk, n)
    fp_new = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), n))
    fp_cur = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), n))
    u1 = ((rng.integers(0, 1 << 24, n) + 1) * 2.0 ** -24)
    if mode in ("delta0", "u1"):
        # choose f'(z) so that Delta hits a target: log ratio = target - beta k (a' - a)
        target = rng.uniform(-2e-4, 2e-4, n) if mode == "delta0" else -rng.exponential(2.0, n)
        one_new, one_cur = 1.0 - a_new ** 2, 1.0 - acur ** 2
        log_ratio = target - bk * (a_new - acur)
        fp_cur = np.sqrt(one_new * fp_new ** 2 / (one_cur * np.exp(2.0 * log_ratio)))
        keep = np.isfinite(fp_cur) & (fp_cur > 1e-6) & (fp_cur < 1e6)
        bk, a_new, acur, fp_new, fp_cur, u1, target = (v[keep] for v in (bk, a_new, acur, fp_new, fp_cur, u1, target))
        if mode == "u1":
            u1 = np.clip(np.exp(target) * (1.0 + rng.uniform(-3e-4, 3e-4, target.size)), 2.0 ** -24, 1.0)
    z = np.zeros_like(bk)
    return np.stack([bk, a_new, acur, fp_new, fp_cur, u1, z, z], axis=1).astype(np.float32)


@pytest.mark.parametrize("mode", ["typical", "delta0", "u1"])
def test_metropolis_screen_agrees_with_exact_test(mode):
    from paper_1010_1486_gb300 import su2

    rng = np.random.default_rng({"typical": 1, "delta0": 2, "u1": 3}[mode])
    q = octuples(rng, 1 << 21, mode)
    screen, exact = su2.su2_selftest_math(5, q)
    assert set(np.unique(screen)) <= {0.0, 1.0, 2.0}
    decided = screen != 2.0
    assert np.array_equal(screen[decided], exact[decided])
    undecided = float(np.mean(~decided))
    if mode == "typical":
        assert undecided < 1e-3
        assert 0.05 < float(np.mean(exact)) < 0.95  # both verdicts occur
    else:
        assert 0.0 < undecided < 1.0  # the band is hit, and not everything falls in it
    # a' = +-1 (zero proposal density factor) and a = +-1 go to the exact rules
    e = q[:256].copy()
    e[:128, 1] = 1.0
    e[128:, 2] = -1.0
    s, x = su2.su2_selftest_math(5, e)
    d = s != 2.0
    assert np.array_equal(s[d], x[d])
