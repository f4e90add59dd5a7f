"""Pins of the oracle's building blocks against things other than itself.

- Philox4x32-10 against PyTorch's independent header-only implementation
  (``at::philox_engine``), compiled here on the host.
- log / exp / sin-cos of 2*pi*u against binary64 numpy, within 2 ulp, over the
  ranges the heat bath uses (Sec. 2: a0 = 1 + ln(x)/(beta k), x in
  [exp(-2 beta k), 1]; direction angle 2*pi*u).
- Quaternion product (Sec. 2, U = a0 + i a.sigma) against 2x2 complex matrices.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _torch_include():
    try:
        import torch  # noqa: F401
    except Exception:
        return None
    import torch.utils.cpp_extension as ce

    for d in ce.include_paths():
        if os.path.exists(os.path.join(d, "ATen", "core", "PhiloxRNGEngine.h")):
            return d
    return None


@pytest.fixture(scope="module")
def torch_philox(tmp_path_factory):
    inc = _torch_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("PyTorch headers or g++ not available")
    exe = str(tmp_path_factory.mktemp("philox") / "philox_torch_pin")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, os.path.join(HERE, "philox_torch_pin.cpp"), "-o", exe],
                   check=True)

    def run(rows):
        text = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
        return np.array([[int(w) for w in line.split()] for line in out.strip().splitlines()], dtype=np.uint64)

    return run


def test_philox_matches_torch_header(torch_philox):
    rng = np.random.default_rng(12345)
    rows = rng.integers(0, 2**32, size=(400, 6), dtype=np.uint64)
    # the counter shapes the heat bath uses, plus edge words
    rows[0] = [1, 0, 0, 0, 0, 0]
    rows[1] = [0, 0, 0, 0, 0, 0]
    rows[2] = [2**32 - 1] * 6
    rows[3] = [3, 0, 1327104, 57, (1 << 3) | (1 << 2) | 3, 2]
    want = torch_philox(rows)
    for r, w in zip(rows, want):
        key = [r[0], r[1]]
        ctr = [r[2], r[3], r[4], r[5]]
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == [int(x) for x in w], (r, got, w)


def test_u01_is_exact_and_in_half_open_unit_interval():
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0
    assert oracle.u01(0x80000000) == 0.5 + 2.0 ** -24
    for x in [1, 255, 256, 12345678, 0xDEADBEEF]:
        assert oracle.u01(x) == ((x >> 8) + 1) * 2.0 ** -24


def test_u01_log_reaches_2_to_minus_33_and_rounds_once():
    """The uniform under a logarithm is w 2^-32 + 2^-33 with w rounded to the
    nearest binary32 first: exact (2w + 1) 2^-33 below 2^23, in [2^-33, 1],
    non-decreasing in w, so -ln x reaches 33 ln 2 = 22.9 instead of the 16.6 of
    a 24-bit uniform (the Creutz proposal of Sec. 2 keeps its tail down to
    beta k (1 - a0) = 22.9)."""
    assert oracle.u01_log(0) == 2.0 ** -33
    assert oracle.u01_log(0xFFFFFFFF) == 1.0
    for x in [1, 2, 1000, (1 << 23) - 1]:
        assert oracle.u01_log(x) == (2 * x + 1) * 2.0 ** -33
    rng = np.random.default_rng(4)
    w = np.sort(rng.integers(0, 1 << 32, 20000, dtype=np.uint64))
    got = np.array([oracle.u01_log(int(x)) for x in w])
    # float32(w) exactly in float64, times 2^-32, plus 2^-33 is exact in float64,
    # so one rounding to float32 reproduces the fused multiply-add
    want = (w.astype(np.float32).astype(np.float64) * 2.0 ** -32 + 2.0 ** -33).astype(np.float32)
    assert np.array_equal(got.astype(np.float32), want)
    assert np.all(np.diff(got) >= 0.0)
    assert -np.log(oracle.u01_log(0)) > 22.8


def _ulp_err(got32, exact64):
    ref32 = np.abs(exact64).astype(np.float32)
    ulp = np.spacing(ref32).astype(np.float64)
    return np.abs(got32.astype(np.float64) - exact64) / ulp


def test_logf_within_2ulp():
    rng = np.random.default_rng(1)
    # random normal floats in [1.2e-38, 1] by bit pattern, plus the region near 1
    bits = rng.integers(0x00800000, 0x3F800001, size=2_000_000, dtype=np.uint32)
    x = bits.view(np.float32)
    near1 = (1.0 - np.arange(1, 200_001, dtype=np.float64) * 2.0 ** -24).astype(np.float32)
    x = np.concatenate([x, near1, np.float32([1.0, 0.5, 2.0 ** -126, 0.70710677, 0.7071068])])
    got = oracle.logf(x)
    exact = np.log(x.astype(np.float64))
    nz = exact != 0
    err = _ulp_err(got[nz], exact[nz])
    assert err.max() <= 2.0, (err.max(), x[nz][np.argmax(err)])
    assert got[x == 1.0][0] == 0.0


def test_expf_within_2ulp():
    rng = np.random.default_rng(2)
    y = np.concatenate([
        rng.uniform(-86.0, 0.0, size=2_000_000),
        -np.arange(0, 100_000) * 1e-6,
        [-86.0, -43.0 * 2, -0.5 * np.log(2), -np.log(2), -1e-30],
    ]).astype(np.float32)
    got = oracle.expf(y)
    exact = np.exp(y.astype(np.float64))
    err = _ulp_err(got, exact)
    assert err.max() <= 2.0, (err.max(), y[np.argmax(err)])
    assert oracle.expf(np.float32([0.0]))[0] == 1.0


def test_sincos2pi_within_2ulp_on_every_uniform():
    # every value the generator can produce: u = m 2^-24, m = 1..2^24
    u = (np.arange(1, 2 ** 24 + 1, dtype=np.float64) * 2.0 ** -24).astype(np.float32)
    s, c = oracle.sincos2pi(u)
    ang = 2.0 * np.pi * u.astype(np.float64)
    for got, exact in ((s, np.sin(ang)), (c, np.cos(ang))):
        big = np.abs(exact) > 1e-6
        err = _ulp_err(got[big], exact[big])
        assert err.max() <= 2.0, err.max()
        # near the zeros: absolute error below 2 ulp of 1e-6
        assert np.abs(got[~big].astype(np.float64) - exact[~big]).max() <= 2 * np.spacing(np.float32(1e-6))
    assert np.abs(s.astype(np.float64) ** 2 + c.astype(np.float64) ** 2 - 1.0).max() < 3e-7


# --------------------------------------------------------------- quaternions
_SIGMA = [np.array([[0, 1], [1, 0]], dtype=complex),
          np.array([[0, -1j], [1j, 0]], dtype=complex),
          np.array([[1, 0], [0, -1]], dtype=complex)]


def to_matrix(a):
    a = np.asarray(a, dtype=np.float64)
    return a[0] * np.eye(2) + 1j * sum(a[i + 1] * _SIGMA[i] for i in range(3))


def from_matrix(m):
    # m = a0 1 + i a.sigma  ->  a0 = Re m00, a3 = Im m00, a2 = Re m01, a1 = Im m01
    return np.array([m[0, 0].real, m[0, 1].imag, m[0, 1].real, m[0, 0].imag])


def test_quaternion_product_is_su2_matrix_product():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a = rng.normal(size=4).astype(np.float32)
        b = rng.normal(size=4).astype(np.float32)
        got = oracle.quat_mul(a, b).astype(np.float64)
        want = from_matrix(to_matrix(a) @ to_matrix(b))
        assert np.allclose(got, want, rtol=0, atol=2e-6 * (1 + np.abs(want).max())), (a, b, got, want)
        # det(U) = |a|^2, trace = 2 a0, dagger is the inverse on S^3
        assert np.isclose(np.linalg.det(to_matrix(a)).real, float(np.dot(a.astype(np.float64), a)), rtol=1e-12)
        assert np.isclose(np.trace(to_matrix(a)).real, 2 * a[0])


def test_quaternion_dagger_inverts_unit_elements():
    rng = np.random.default_rng(4)
    for _ in range(200):
        a = rng.normal(size=4)
        a = (a / np.linalg.norm(a)).astype(np.float32)
        d = np.array([a[0], -a[1], -a[2], -a[3]], dtype=np.float32)
        assert np.allclose(oracle.quat_mul(a, d), [1, 0, 0, 0], atol=3e-7)
        m = to_matrix(a)
        assert np.allclose(m @ m.conj().T, np.eye(2), atol=1e-6)


def log_uniforms(w):
    """r1 as the definition draws it for a logarithm: the word rounded to
    binary32, times 2^-32, plus 2^-33, rounded once (exact in binary64
    before the last rounding)."""
    w = np.asarray(w, dtype=np.uint64)
    return (w.astype(np.float32).astype(np.float64) * 2.0 ** -32 + 2.0 ** -33).astype(np.float32)


def cutoff_words():
    """The smallest words (r1 down to 2^-33, where x = e + r1 (1 - e) is most
    sensitive to e), the largest, and random ones."""
    rng = np.random.default_rng(0)
    return np.concatenate([np.arange(0, 4097), np.arange(2 ** 32 - 4096, 2 ** 32),
                           rng.integers(0, 2 ** 32, 50_000)]).astype(np.uint32)


def test_log_uniform_is_the_whole_word_rounded_once():
    w = cutoff_words()
    r1, _ = oracle.creutz_x_a0(np.full(w.size, 50.0, np.float32), w)  # e = 0 above 43
    assert np.array_equal(r1, log_uniforms(w))
    assert r1.min() == np.float32(2.0 ** -33) and r1.max() == np.float32(1.0)


def test_creutz_variable_ignores_exp_above_21():
    """The heat-bath kernels do not compute e = exp(-2 beta k) above
    beta k = 21 and take x = r1; the definition keeps e up to 43.  This is
    the same draw only if x = r1 (1 - e) + e rounds to r1 for every log
    uniform r1 >= 2^-33 there: e < exp(-42) < 2^-60 lies below half an ulp
    of 2^-33 (2^-57).  Checked on the definition's own x for the smallest,
    the largest and random words over beta k in (21, 43], and against a
    cutoff of 17, which moves x for the smallest words."""
    assert float(oracle.expf(np.array([-42.0], np.float32))[0]) < 2.0 ** -60
    w = cutoff_words()
    r1 = log_uniforms(w)
    bks = np.concatenate([[np.nextafter(np.float32(21.0), np.float32(50.0))],
                          np.linspace(21.0, 43.0, 221)[1:], [np.float32(43.0)]]).astype(np.float32)
    for bk in bks:
        x, _ = oracle.creutz_x_a0(np.full(w.size, bk, np.float32), w)
        assert np.array_equal(x, r1), bk
    # at beta k = 17.5 the smallest words do move: x = r1 is not the definition there
    x, _ = oracle.creutz_x_a0(np.full(w.size, 17.5, np.float32), w)
    moved = w[x != r1]
    assert moved.size > 0 and moved.max() < 2 ** 12, moved[:8]
    assert x[1] != r1[1]  # w = 1: r1 = 3.49246e-10, x = 3.492466e-10
    # the smallest beta k from which no word moves lies between 19.5 and 21
    lo = np.float32(19.5)
    x, _ = oracle.creutz_x_a0(np.full(w.size, lo, np.float32), w)
    assert not np.array_equal(x, r1)
