"""su2_plaquette_noalloc: the mean plaquette for callers that cannot allocate
device memory (their framework owns all of it, or an allocation is not allowed
where they call).  It reads caller-provided device links, writes a
caller-provided device double, and keeps its reduction scratch in a fixed
array inside the library.  Checked through the C ABI against su2_plaquette
and against the CPU oracle's plaquette of the same links, on two calls in a
row (which reuse that shared scratch).  This file is collected last so that a
run stopping at the first failure has run every other test."""
import ctypes

import pytest

import oracle
from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu

OBS_REL = 1e-6  # the tolerance of the plaquette parity tests


def _close(got, want):
    return abs(got - want) <= OBS_REL * max(abs(want), 0.05)


def test_noalloc_plaquette_matches_su2_plaquette_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    shapes = [(8, 6, 2.3, 7), (6, 4, 1.9, 8)]
    lats = []
    try:
        for ns, nt, beta, seed in shapes:
            h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT)
            lats.append(h)
            su2.su2_heatbath_sweep(h, 2)
        want = [su2.su2_plaquette(h) for h in lats]
        ref = [oracle.plaquette(ns, nt, su2.su2_get_links(h, ns, nt)) for (ns, nt, _, _), h in zip(shapes, lats)]
        # output buffer owned by the caller; the entry point allocates nothing
        out = torch.full((2,), -7.0, dtype=torch.float64, device="cuda")
        for k, ((ns, nt, _, _), h) in enumerate(zip(shapes, lats)):
            ptr, _ = su2.su2_device_links(h)
            su2.su2_plaquette_noalloc(ptr, ns, nt, out.data_ptr() + 8 * k, None)
        torch.cuda.synchronize()
        got = out.cpu().tolist()
        for g, w, r in zip(got, want, ref):
            assert _close(g, w), (got, want)
            assert _close(g, r), (got, ref)
        # the same lattice twice more in a row: the shared scratch starts clean each time
        ptr, _ = su2.su2_device_links(lats[0])
        su2.su2_plaquette_noalloc(ptr, 8, 6, out.data_ptr(), None)
        su2.su2_plaquette_noalloc(ptr, 8, 6, out.data_ptr() + 8, None)
        torch.cuda.synchronize()
        again = out.cpu().tolist()
        assert _close(again[0], want[0]) and _close(again[1], want[0]), (again, want)
        assert _close(again[0], ref[0]) and _close(again[1], ref[0]), (again, ref)
    finally:
        for h in lats:
            su2.su2_destroy(h)


def test_noalloc_plaquette_rejects_sizes_beyond_its_scratch():
    lib = su2.library()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert lib.su2_plaquette_noalloc(dummy, 96, 96, dummy, None) == 1
    assert "67108864" in su2.su2_last_error()
    assert lib.su2_plaquette_noalloc(dummy, 7, 8, dummy, None) == 1
    assert lib.su2_plaquette_noalloc(None, 8, 8, dummy, None) == 1
