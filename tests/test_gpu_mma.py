"""Tensor-core (tcgen05) self-test: BF16 x BF16 -> FP32 products against the
exact product of the same BF16 values on the host."""
import numpy as np
import pytest

from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu


def to_bf16_bits(x):
    """Round-to-nearest-even BF16 of float32 values, as uint16 bits."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def bf16_to_f32(b):
    return (b.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("k", [16, 32])
def test_tcgen05_bf16_gemm(k):
    rng = np.random.default_rng(k)
    a = to_bf16_bits(rng.normal(size=(128, k)))
    b = to_bf16_bits(rng.normal(size=(32, k)))
    d = su2.su2_selftest_mma(a, b)
    want = bf16_to_f32(a).astype(np.float64) @ bf16_to_f32(b).astype(np.float64).T
    assert np.allclose(d, want, rtol=1e-5, atol=1e-5), np.abs(d - want).max()
