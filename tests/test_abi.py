"""The C-ABI library builds, loads and exports every function that
include/su2.h declares; host-side argument checks need no GPU."""
import ctypes
import math

import pytest

from paper_1010_1486_gb300 import _build


@pytest.fixture(scope="module")
def su2():
    try:
        _build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    _build.build()
    from paper_1010_1486_gb300 import su2 as mod

    return mod


def test_every_declared_symbol_is_exported(su2):
    names = su2.declared_symbols()
    assert len(names) >= 20
    lib = ctypes.CDLL(su2.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    core = {"su2_create", "su2_destroy", "su2_heatbath_sweep", "su2_reunitarize", "su2_plaquette", "su2_polyakov"}
    assert core <= set(names)
    assert su2.su2_abi_version() == 3
    # su2_stats as declared: 8 + 8 + 8*8 + 8 + 4 + 4 + 8 + 8 + 8 + 8 bytes
    assert ctypes.sizeof(su2.su2_stats) == 128


@pytest.mark.parametrize("ns,nt", [(3, 4), (4, 3), (0, 4), (4, 0), (1, 2), (-2, 4), (2000, 2000), (150, 160),
                                   (64, 2048)])  # 4V = 2^31 exactly: one past the largest lattice
def test_create_rejects_bad_extents(su2, ns, nt):
    with pytest.raises(su2.SU2Error) as e:
        su2.su2_create(ns, nt, 2.3, 1)
    assert e.value.status == 1


@pytest.mark.parametrize("beta", [-1.0, math.nan, math.inf, -math.inf])
def test_create_rejects_bad_beta(su2, beta):
    with pytest.raises(su2.SU2Error) as e:
        su2.su2_create(4, 4, beta, 1)
    assert e.value.status == 1


def test_null_and_enum_arguments(su2):
    lib = su2.library()
    assert lib.su2_create(4, 4, 2.3, 1, 0, None, None) == 1
    h = ctypes.c_void_p()
    assert lib.su2_create(4, 4, 2.3, 1, 7, None, ctypes.byref(h)) == 1
    assert lib.su2_get_state(None, None) == 1
    assert lib.su2_plaquette(None, None) == 1
    assert lib.su2_heatbath_sweep(None, 1, None) == 1
    assert lib.su2_overrelax_sweep(None, 1) == 1
    assert lib.su2_overrelax_phase(None, 0, 0) == 1
    assert lib.su2_set_overrelax(None, 1) == 1
    assert lib.su2_wilson_loops(None, 1, 1, None) == 1
    out = ctypes.c_uint()
    assert lib.su2_selftest_mbar_timeout(0, 100, ctypes.byref(out)) == 1
    assert lib.su2_selftest_mbar_timeout(8, 0, ctypes.byref(out)) == 1
    assert lib.su2_selftest_mbar_timeout(8, (1 << 24) + 1, ctypes.byref(out)) == 1
    assert lib.su2_selftest_mbar_timeout(8, 100, None) == 1
    assert lib.su2_destroy(None) == 0
    # allocator hooks must come in pairs
    assert lib.su2_set_allocator(su2.ALLOC_FN(lambda *a: None), su2.FREE_FN(), None) == 1
    assert lib.su2_set_allocator(su2.ALLOC_FN(), su2.FREE_FN(), None) == 0


def test_status_strings(su2):
    for code in range(8):
        assert su2.su2_status_str(code)
    assert su2.su2_status_str(0) == "ok"


def test_no_silent_fallback_without_a_gpu(su2):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(su2.SU2Error) as e:
        su2.su2_create(4, 4, 2.3, 1)
    assert e.value.status == 3  # SU2_E_CUDA: fails loudly, computes nothing on the host
