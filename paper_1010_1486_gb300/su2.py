"""Thin Python binding of the ``libsu2`` C ABI (``include/su2.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libsu2.so``.  Functions carry the C names; a non-OK status raises
:class:`SU2Error`.  If the library has not been built, importing this module
raises ``ImportError`` -- there is no fallback of any kind.

PyTorch supplies device memory and streams: :func:`use_torch_allocator`
routes the library's device allocations through PyTorch's caching allocator,
and ``stream`` arguments accept a ``torch.cuda.Stream`` or a raw handle.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsu2.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "su2.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

SU2_COLD, SU2_HOT = 0, 1
SU2_SAMPLER_CREUTZ, SU2_SAMPLER_KP = 0, 1
STATUS = {0: "SU2_OK", 1: "SU2_E_INVAL", 2: "SU2_E_NOMEM", 3: "SU2_E_CUDA", 4: "SU2_E_SAMPLER",
          5: "SU2_E_DEVICE_TIMEOUT", 6: "SU2_E_NUMERIC", 7: "SU2_E_STATE"}


class SU2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = _lib.su2_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_lib.su2_status_str(status).decode()}) {detail}")


class su2_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_uint64), ("link_updates", ctypes.c_uint64),
                ("trials", ctypes.c_uint64 * 8), ("sampler_failures", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint32), ("timed", ctypes.c_uint32),
                ("kernel_ms", ctypes.c_double), ("overrelax_sweeps", ctypes.c_uint64),
                ("overrelax_updates", ctypes.c_uint64), ("overrelax_ms", ctypes.c_double)]

    def as_dict(self):
        return {"sweeps": self.sweeps, "link_updates": self.link_updates, "trials": list(self.trials),
                "sampler_failures": self.sampler_failures, "kernel_launches": self.kernel_launches,
                "timed": bool(self.timed), "kernel_ms": self.kernel_ms,
                "overrelax_sweeps": self.overrelax_sweeps, "overrelax_updates": self.overrelax_updates,
                "overrelax_ms": self.overrelax_ms}


class su2_learned_stats(ctypes.Structure):
    _fields_ = [("link_updates", ctypes.c_uint64), ("accepted", ctypes.c_uint64 * 8),
                ("plain_trials", ctypes.c_uint64 * 8), ("learned_sweeps", ctypes.c_uint32),
                ("plain_sweeps", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint32),
                ("timed", ctypes.c_uint32), ("kernel_ms", ctypes.c_double)]

    def as_dict(self):
        return {"link_updates": self.link_updates, "accepted": list(self.accepted),
                "plain_trials": list(self.plain_trials), "learned_sweeps": self.learned_sweeps,
                "plain_sweeps": self.plain_sweeps, "kernel_launches": self.kernel_launches,
                "timed": bool(self.timed), "kernel_ms": self.kernel_ms}


class su2_state(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int32), ("nt", ctypes.c_int32), ("beta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("sweep", ctypes.c_uint32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)

_P = ctypes.c_void_p
_i32, _u32, _u64, _f64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
_SIGS = {
    "su2_set_allocator": [ALLOC_FN, FREE_FN, _P],
    "su2_create": [_i32, _i32, _f64, _u64, _i32, _P, ctypes.POINTER(_P)],
    "su2_destroy": [_P],
    "su2_heatbath_sweep": [_P, _i32, ctypes.POINTER(su2_stats)],
    "su2_heatbath_phase": [_P, _i32, _i32],
    "su2_generate": [_P, _i32, _i32, _i32, _P, _P, ctypes.POINTER(su2_stats)],
    "su2_reunitarize": [_P],
    "su2_plaquette": [_P, ctypes.POINTER(_f64)],
    "su2_polyakov": [_P, ctypes.POINTER(_f64)],
    "su2_get_links": [_P, _P],
    "su2_set_links": [_P, _P],
    "su2_get_links_async": [_P, _P],
    "su2_set_links_async": [_P, _P],
    "su2_generate_async": [_P, _i32, _i32, _i32, _P, _P],
    "su2_sync": [_P],
    "su2_check_links": [_P, _f64, ctypes.POINTER(_u64), ctypes.POINTER(_u64)],
    "su2_set_trial_cap": [_P, _i32],
    "su2_get_state": [_P, ctypes.POINTER(su2_state)],
    "su2_set_state": [_P, ctypes.POINTER(su2_state)],
    "su2_set_beta": [_P, _f64],
    "su2_device_links": [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t)],
    "su2_set_timing": [_P, _i32],
    "su2_set_sampler": [_P, _i32],
    "su2_overrelax_sweep": [_P, _i32],
    "su2_wilson_loops": [_P, _i32, _i32, _P],
    "su2_overrelax_phase": [_P, _i32, _i32],
    "su2_set_overrelax": [_P, _i32],
    "su2_selftest_philox": [_P, _P, ctypes.c_size_t],
    "su2_selftest_math": [_i32, _P, _P, _P, ctypes.c_size_t],
    "su2_plaquette_noalloc": [_P, _i32, _i32, _P, _P],
    "su2_batch_create": [_i32, _P, _P, _P, _P, _i32, _P, ctypes.POINTER(_P)],
    "su2_batch_destroy": [_P],
    "su2_batch_sweep": [_P, _i32, ctypes.POINTER(su2_stats)],
    "su2_batch_generate": [_P, _i32, _i32, _P, _P, ctypes.POINTER(su2_stats)],
    "su2_batch_plaquette": [_P, _P],
    "su2_batch_polyakov": [_P, _P],
    "su2_batch_get_links": [_P, _i32, _P],
    "su2_batch_set_config": [_P, _i32, _i32],
    "su2_batch_set_launch": [_P, _i32, _i32, _i32],
    "su2_batch_set_sampler": [_P, _i32],
    "su2_batch_launch_info": [_P, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
    "su2_batch_autotune": [_P, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
    "su2_batch_info": [_P, ctypes.POINTER(_i32), ctypes.POINTER(_u32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                       ctypes.POINTER(_i32)],
    "su2_selftest_barrier_timeout": [_i32, _u64, ctypes.POINTER(_u32)],
    "su2_selftest_mbar_timeout": [_i32, _u32, ctypes.POINTER(_u32)],
    "su2_selftest_mma": [_P, _P, _i32, _P],
    "su2_set_proposal": [_P, _P, _i32, _f64, _f64, _i32],
    "su2_get_proposal_table": [_P, _P],
    "su2_learned_generate": [_P, _i32, _i32, _f64, _P, _P, ctypes.POINTER(su2_learned_stats)],
    "su2_learned_sweep": [_P, _i32, ctypes.POINTER(su2_learned_stats)],
    "su2_slab_create": [_i32, _i32, _i32, _i32, _f64, _u64, _i32, _P, ctypes.POINTER(_P)],
    "su2_slab_destroy": [_P],
    "su2_slab_set_sampler": [_P, _i32],
    "su2_slab_phase": [_P, _i32, _i32],
    "su2_slab_pack": [_P, _i32, _i32, _i32, _P],
    "su2_slab_unpack": [_P, _i32, _i32, _i32, _P],
    "su2_slab_exchange": [_P, _P, _i32, _i32],
    "su2_slab_sync": [_P],
    "su2_slab_get_links": [_P, _P],
    "su2_slab_set_links": [_P, _P],
    "su2_slab_stats": [_P, _P, ctypes.POINTER(_u64)],
    "su2_slab_info": [_P, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_u32)],
    "su2_collect_pairs": [_P, _i32, _i32, _i32, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "su2_trainer_create": [_P, _u64, _P, ctypes.POINTER(_P)],
    "su2_trainer_destroy": [_P],
    "su2_trainer_set_input_scaling": [_P, _P, ctypes.c_size_t],
    "su2_trainer_fit": [_P, _P, ctypes.c_size_t, _i32, _i32, _f64, _P],
    "su2_trainer_gradient": [_P, _P, ctypes.c_size_t, ctypes.POINTER(_f64), _P],
    "su2_trainer_get_weights": [_P, _P],
}
for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_int
_lib.su2_status_str.argtypes = [ctypes.c_int]
_lib.su2_status_str.restype = ctypes.c_char_p
_lib.su2_last_error.argtypes = []
_lib.su2_last_error.restype = ctypes.c_char_p
_lib.su2_abi_version.argtypes = []
_lib.su2_abi_version.restype = ctypes.c_int
_lib.su2_slab_boundary_bytes.argtypes = [_P]
_lib.su2_slab_boundary_bytes.restype = ctypes.c_size_t


def declared_symbols() -> list[str]:
    """Function names declared in include/su2.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(su2_\w+)\s*\(", text, flags=re.M)))


def library():
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise SU2Error(status, where)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def _host_ptr(a: np.ndarray) -> int:
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host buffer must be C-contiguous")
    return a.ctypes.data


# --------------------------------------------------------------- allocator
_torch_hooks = None


def use_torch_allocator() -> None:
    """Route device allocations through PyTorch's caching allocator."""
    global _torch_hooks
    import torch

    def _alloc(nbytes, device, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device), stream=int(stream or 0)))
        except Exception:
            return None

    def _free(ptr, nbytes, device, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(_lib.su2_set_allocator(hooks[0], hooks[1], None), "su2_set_allocator")
    _torch_hooks = hooks


def use_default_allocator() -> None:
    global _torch_hooks
    _check(_lib.su2_set_allocator(ALLOC_FN(), FREE_FN(), None), "su2_set_allocator")
    _torch_hooks = None


# ------------------------------------------------------------------ C names
def su2_create(ns: int, nt: int, beta: float, seed: int, start: int = SU2_HOT, stream=None) -> int:
    h = _P()
    _check(_lib.su2_create(ns, nt, float(beta), int(seed), int(start), _stream_handle(stream), ctypes.byref(h)),
           "su2_create")
    return h.value


def su2_destroy(lat: int) -> None:
    _check(_lib.su2_destroy(lat), "su2_destroy")


def su2_heatbath_sweep(lat: int, nsweeps: int = 1, stats: bool = False):
    st = su2_stats() if stats else None
    _check(_lib.su2_heatbath_sweep(lat, nsweeps, ctypes.byref(st) if st is not None else None),
           "su2_heatbath_sweep")
    return st.as_dict() if st is not None else None


def su2_heatbath_phase(lat: int, mu: int, parity: int) -> None:
    _check(_lib.su2_heatbath_phase(lat, mu, parity), "su2_heatbath_phase")


def su2_generate(lat: int, nsweeps: int, measure_every: int = 1, reunit_every: int = 0,
                 plaq: np.ndarray | None = None, poly: np.ndarray | None = None):
    """Returns (plaquettes, polyakov loops, stats dict).  plaq / poly may be
    caller-provided float64 arrays (e.g. pinned host memory)."""
    nmeas = nsweeps // measure_every if measure_every > 0 else 0
    if plaq is None:
        plaq = np.zeros(nmeas, dtype=np.float64)
    if poly is None:
        poly = np.zeros(nmeas, dtype=np.float64)
    st = su2_stats()
    _check(_lib.su2_generate(lat, nsweeps, measure_every, reunit_every, _host_ptr(plaq) if nmeas else None,
                             _host_ptr(poly) if nmeas else None, ctypes.byref(st)), "su2_generate")
    return plaq[:nmeas], poly[:nmeas], st.as_dict()


def su2_reunitarize(lat: int) -> None:
    _check(_lib.su2_reunitarize(lat), "su2_reunitarize")


def su2_plaquette(lat: int) -> float:
    out = _f64()
    _check(_lib.su2_plaquette(lat, ctypes.byref(out)), "su2_plaquette")
    return out.value


def su2_polyakov(lat: int) -> float:
    out = _f64()
    _check(_lib.su2_polyakov(lat, ctypes.byref(out)), "su2_polyakov")
    return out.value


def su2_get_links(lat: int, ns: int, nt: int, out: np.ndarray | None = None) -> np.ndarray:
    """Links as float32 [site, mu, 4] in lexicographic site order."""
    if out is None:
        out = np.empty((ns ** 3 * nt, 4, 4), dtype=np.float32)
    _check(_lib.su2_get_links(lat, _host_ptr(out)), "su2_get_links")
    return out


def su2_set_links(lat: int, links: np.ndarray) -> None:
    links = np.ascontiguousarray(links, dtype=np.float32)
    _check(_lib.su2_set_links(lat, _host_ptr(links)), "su2_set_links")


def su2_set_links_async(lat: int, links: np.ndarray) -> None:
    """Enqueues the upload of `links` (C-contiguous float32 [site, mu, 4]);
    the caller keeps the array alive and unchanged until su2_sync."""
    if not (links.flags["C_CONTIGUOUS"] and links.dtype == np.float32):
        raise ValueError("su2_set_links_async needs a C-contiguous float32 array")
    _check(_lib.su2_set_links_async(lat, _host_ptr(links)), "su2_set_links_async")


def su2_get_links_async(lat: int, out: np.ndarray) -> None:
    """Enqueues the download of the links into `out` (C-contiguous float32
    [site, mu, 4]), valid after su2_sync."""
    if not (out.flags["C_CONTIGUOUS"] and out.dtype == np.float32):
        raise ValueError("su2_get_links_async needs a C-contiguous float32 array")
    _check(_lib.su2_get_links_async(lat, _host_ptr(out)), "su2_get_links_async")


def su2_generate_async(lat: int, nsweeps: int, measure_every: int = 1, reunit_every: int = 0,
                       plaq: np.ndarray | None = None, poly: np.ndarray | None = None) -> None:
    """su2_generate without statistics and without waiting; plaq / poly
    (float64, nsweeps // measure_every values, nullable) hold their values
    after su2_sync."""
    nmeas = nsweeps // measure_every if measure_every > 0 else 0
    for a in (plaq, poly):
        if a is not None and (a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size < nmeas):
            raise ValueError("su2_generate_async: plaq / poly need nsweeps // measure_every float64 values")
    _check(_lib.su2_generate_async(lat, nsweeps, measure_every, reunit_every,
                                   _host_ptr(plaq) if plaq is not None and nmeas else None,
                                   _host_ptr(poly) if poly is not None and nmeas else None), "su2_generate_async")


def su2_sync(lat: int) -> None:
    _check(_lib.su2_sync(lat), "su2_sync")


def su2_check_links(lat: int, tol: float = 1e-6):
    """(non-finite links, links with | |a| - 1 | > tol); raises SU2Error
    (SU2_E_NUMERIC) if any link is non-finite."""
    nf, off = _u64(), _u64()
    _check(_lib.su2_check_links(lat, float(tol), ctypes.byref(nf), ctypes.byref(off)), "su2_check_links")
    return nf.value, off.value


def su2_set_trial_cap(lat: int, max_trials: int) -> None:
    _check(_lib.su2_set_trial_cap(lat, int(max_trials)), "su2_set_trial_cap")


def su2_get_state(lat: int) -> dict:
    s = su2_state()
    _check(_lib.su2_get_state(lat, ctypes.byref(s)), "su2_get_state")
    return {"ns": s.ns, "nt": s.nt, "beta": s.beta, "seed": s.seed, "sweep": s.sweep}


def su2_set_state(lat: int, state: dict) -> None:
    s = su2_state(state["ns"], state["nt"], state["beta"], state["seed"], state["sweep"])
    _check(_lib.su2_set_state(lat, ctypes.byref(s)), "su2_set_state")


def su2_set_beta(lat: int, beta: float) -> None:
    _check(_lib.su2_set_beta(lat, float(beta)), "su2_set_beta")


def su2_device_links(lat: int):
    p = _P()
    n = ctypes.c_size_t()
    _check(_lib.su2_device_links(lat, ctypes.byref(p), ctypes.byref(n)), "su2_device_links")
    return p.value, n.value


def su2_set_sampler(lat: int, sampler: int) -> None:
    _check(_lib.su2_set_sampler(lat, int(sampler)), "su2_set_sampler")


def su2_wilson_loops(lat: int, rmax: int, tmax: int) -> np.ndarray:
    """W[R-1, T-1], the mean (1/2) Tr of the R x T space-time Wilson loops."""
    out = np.zeros(rmax * tmax, dtype=np.float64)
    _check(_lib.su2_wilson_loops(lat, rmax, tmax, out.ctypes.data_as(ctypes.c_void_p)), "su2_wilson_loops")
    return out.reshape(rmax, tmax)


def su2_overrelax_sweep(lat: int, nsweeps: int = 1) -> None:
    _check(_lib.su2_overrelax_sweep(lat, nsweeps), "su2_overrelax_sweep")


def su2_overrelax_phase(lat: int, mu: int, parity: int) -> None:
    _check(_lib.su2_overrelax_phase(lat, mu, parity), "su2_overrelax_phase")


def su2_set_overrelax(lat: int, n_or: int) -> None:
    _check(_lib.su2_set_overrelax(lat, int(n_or)), "su2_set_overrelax")


def su2_set_timing(lat: int, enable: bool) -> None:
    _check(_lib.su2_set_timing(lat, int(bool(enable))), "su2_set_timing")


def su2_selftest_philox(ck: np.ndarray) -> np.ndarray:
    ck = np.ascontiguousarray(ck, dtype=np.uint32).reshape(-1, 6)
    out = np.zeros((ck.shape[0], 4), dtype=np.uint32)
    _check(_lib.su2_selftest_philox(_host_ptr(ck), _host_ptr(out), ck.shape[0]), "su2_selftest_philox")
    return out


def su2_selftest_math(which: int, x: np.ndarray):
    """which = 4 takes x of shape (n, 4): rows (r1, r2, 1/(beta k), exp(-2 beta k));
    which = 5 x of shape (n, 8): rows (beta k, a', a, f'(z'), f'(z), u1, 0, 0);
    which = 6 x of shape (n, 2): rows (beta k, Philox word bits as float32)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n = x.shape[0] if which in (4, 5, 6) else x.size
    y = np.empty(n, dtype=np.float32)
    y2 = np.empty(n, dtype=np.float32) if which in (2, 4, 5, 6) else None
    _check(_lib.su2_selftest_math(which, _host_ptr(x), _host_ptr(y), _host_ptr(y2) if y2 is not None else None,
                                  n), "su2_selftest_math")
    if which not in (4, 5, 6):
        y = y.reshape(x.shape)
        y2 = y2.reshape(x.shape) if y2 is not None else None
    return (y, y2) if y2 is not None else y


def su2_plaquette_noalloc(links_ptr: int, ns: int, nt: int, out_ptr: int, stream=None) -> None:
    """Mean plaquette of device-resident links (even/odd layout of
    su2_device_links) into the device double at out_ptr, allocating nothing.
    For callers that cannot allocate device memory at this point; see
    include/su2.h for the scratch it shares between calls and its size limit."""
    _check(_lib.su2_plaquette_noalloc(links_ptr, ns, nt, out_ptr, _stream_handle(stream)), "su2_plaquette_noalloc")


# --------------------------------------------------------- learned proposal
N_WEIGHTS = 1947
N_SPLINE = 27


def su2_set_proposal(lat: int, weights: np.ndarray, s_lo: float, s_hi: float, grid_points: int = 256) -> None:
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(_lib.su2_set_proposal(lat, _host_ptr(w), w.size, float(s_lo), float(s_hi), int(grid_points)),
           "su2_set_proposal")


def su2_get_proposal_table(lat: int, grid_points: int) -> np.ndarray:
    out = np.zeros((grid_points, N_SPLINE), dtype=np.float32)
    _check(_lib.su2_get_proposal_table(lat, _host_ptr(out)), "su2_get_proposal_table")
    return out


def su2_learned_generate(lat: int, nsweeps: int, measure_every: int = 1, min_acceptance: float = 0.7,
                         plaq: np.ndarray | None = None, poly: np.ndarray | None = None):
    nmeas = nsweeps // measure_every if measure_every > 0 else 0
    if plaq is None:
        plaq = np.zeros(max(nmeas, 1), dtype=np.float64)
    if poly is None:
        poly = np.zeros(max(nmeas, 1), dtype=np.float64)
    st = su2_learned_stats()
    _check(_lib.su2_learned_generate(lat, nsweeps, measure_every, float(min_acceptance), _host_ptr(plaq),
                                     _host_ptr(poly), ctypes.byref(st)), "su2_learned_generate")
    return plaq[:nmeas], poly[:nmeas], st.as_dict()


def su2_learned_sweep(lat: int, nsweeps: int):
    """nsweeps learned sweeps, fallback below acceptance 0.7, no measurements."""
    st = su2_learned_stats()
    _check(_lib.su2_learned_sweep(lat, nsweeps, ctypes.byref(st)), "su2_learned_sweep")
    return st.as_dict()


# ------------------------------------------------------------ time slabs
def su2_slab_create(ns: int, nt: int, t0: int, nt_local: int, beta: float, seed: int, start: int = 1,
                    stream=None) -> int:
    h = _P()
    _check(_lib.su2_slab_create(ns, nt, t0, nt_local, float(beta), int(seed), int(start), _stream_handle(stream),
                                ctypes.byref(h)), "su2_slab_create")
    return h.value


def su2_slab_destroy(h: int) -> None:
    _check(_lib.su2_slab_destroy(h), "su2_slab_destroy")


def su2_slab_set_sampler(h: int, sampler: int) -> None:
    _check(_lib.su2_slab_set_sampler(h, int(sampler)), "su2_slab_set_sampler")


def su2_slab_phase(h: int, mu: int, parity: int) -> None:
    _check(_lib.su2_slab_phase(h, mu, parity), "su2_slab_phase")


def su2_slab_boundary_bytes(h: int) -> int:
    return int(_lib.su2_slab_boundary_bytes(h))


def su2_slab_pack(h: int, mu: int, parity: int, side: int, dst_ptr: int) -> None:
    _check(_lib.su2_slab_pack(h, mu, parity, side, dst_ptr), "su2_slab_pack")


def su2_slab_unpack(h: int, mu: int, parity: int, side: int, src_ptr: int) -> None:
    _check(_lib.su2_slab_unpack(h, mu, parity, side, src_ptr), "su2_slab_unpack")


def su2_slab_exchange(lower: int, upper: int, mu: int, parity: int) -> None:
    _check(_lib.su2_slab_exchange(lower, upper, mu, parity), "su2_slab_exchange")


def su2_slab_sync(h: int) -> None:
    _check(_lib.su2_slab_sync(h), "su2_slab_sync")


def su2_slab_get_links(h: int, ns: int, nt_local: int) -> np.ndarray:
    out = np.empty((ns ** 3 * (nt_local + 2), 4, 4), dtype=np.float32)
    _check(_lib.su2_slab_get_links(h, _host_ptr(out)), "su2_slab_get_links")
    return out


def su2_slab_set_links(h: int, links: np.ndarray) -> None:
    links = np.ascontiguousarray(links, dtype=np.float32)
    _check(_lib.su2_slab_set_links(h, _host_ptr(links)), "su2_slab_set_links")


def su2_slab_stats(h: int):
    trials = np.zeros(8, dtype=np.uint64)
    fails = _u64()
    _check(_lib.su2_slab_stats(h, _host_ptr(trials), ctypes.byref(fails)), "su2_slab_stats")
    return [int(t) for t in trials], int(fails.value)


def su2_slab_info(h: int):
    t0, ntl, sw = _i32(), _i32(), _u32()
    _check(_lib.su2_slab_info(h, ctypes.byref(t0), ctypes.byref(ntl), ctypes.byref(sw)), "su2_slab_info")
    return t0.value, ntl.value, sw.value


def su2_collect_pairs(lat: int, mu: int, parity: int, stride: int, dev_ptr: int, cap: int) -> int:
    """(beta k, a0) float2 pairs into the device buffer at dev_ptr (cap pairs)."""
    n = ctypes.c_size_t()
    _check(_lib.su2_collect_pairs(lat, mu, parity, stride, dev_ptr, cap, ctypes.byref(n)), "su2_collect_pairs")
    return n.value


def su2_trainer_create(init_weights: np.ndarray, seed: int = 0, stream=None) -> int:
    w = np.ascontiguousarray(init_weights, dtype=np.float32)
    if w.size != N_WEIGHTS:
        raise ValueError("1947 weights expected")
    h = _P()
    _check(_lib.su2_trainer_create(_host_ptr(w), int(seed), _stream_handle(stream), ctypes.byref(h)),
           "su2_trainer_create")
    return h.value


def su2_trainer_destroy(tr: int) -> None:
    _check(_lib.su2_trainer_destroy(tr), "su2_trainer_destroy")


def su2_trainer_set_input_scaling(tr: int, dev_pairs: int, n: int) -> None:
    _check(_lib.su2_trainer_set_input_scaling(tr, dev_pairs, n), "su2_trainer_set_input_scaling")


def su2_trainer_fit(tr: int, dev_pairs: int, n: int, steps: int, batch: int = 4096, lr: float = 1e-3) -> np.ndarray:
    losses = np.zeros(max(steps, 1), dtype=np.float32)
    _check(_lib.su2_trainer_fit(tr, dev_pairs, n, steps, batch, float(lr), _host_ptr(losses)), "su2_trainer_fit")
    return losses[:steps]


def su2_trainer_gradient(tr: int, dev_pairs: int, n: int):
    loss = _f64()
    grad = np.zeros(1945, dtype=np.float32)
    _check(_lib.su2_trainer_gradient(tr, dev_pairs, n, ctypes.byref(loss), _host_ptr(grad)), "su2_trainer_gradient")
    return loss.value, grad


def su2_trainer_get_weights(tr: int) -> np.ndarray:
    w = np.zeros(N_WEIGHTS, dtype=np.float32)
    _check(_lib.su2_trainer_get_weights(tr, _host_ptr(w)), "su2_trainer_get_weights")
    return w


# ------------------------------------------------------------------ batches
def su2_batch_create(ns, nt, beta, seed, start: int = SU2_COLD, stream=None) -> int:
    n = len(ns)
    a_ns = np.ascontiguousarray(ns, dtype=np.int32)
    a_nt = np.ascontiguousarray(nt, dtype=np.int32)
    a_beta = np.ascontiguousarray(beta, dtype=np.float64)
    a_seed = np.ascontiguousarray(seed, dtype=np.uint64)
    h = _P()
    _check(_lib.su2_batch_create(n, _host_ptr(a_ns), _host_ptr(a_nt), _host_ptr(a_beta), _host_ptr(a_seed),
                                 int(start), _stream_handle(stream), ctypes.byref(h)), "su2_batch_create")
    return h.value


def su2_batch_destroy(b: int) -> None:
    _check(_lib.su2_batch_destroy(b), "su2_batch_destroy")


def su2_batch_sweep(b: int, nsweeps: int = 1) -> dict:
    st = su2_stats()
    _check(_lib.su2_batch_sweep(b, nsweeps, ctypes.byref(st)), "su2_batch_sweep")
    return st.as_dict()


def su2_batch_generate(b: int, n: int, nsweeps: int, measure_every: int = 1):
    """Returns (plaquettes [nmeas, n], Polyakov loops [nmeas, n], stats)."""
    nmeas = nsweeps // measure_every if measure_every > 0 else 0
    plaq = np.zeros((max(nmeas, 1), n), dtype=np.float64)
    poly = np.zeros((max(nmeas, 1), n), dtype=np.float64)
    st = su2_stats()
    _check(_lib.su2_batch_generate(b, nsweeps, measure_every, _host_ptr(plaq), _host_ptr(poly), ctypes.byref(st)),
           "su2_batch_generate")
    return plaq[:nmeas], poly[:nmeas], st.as_dict()


def su2_batch_plaquette(b: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _check(_lib.su2_batch_plaquette(b, _host_ptr(out)), "su2_batch_plaquette")
    return out


def su2_batch_polyakov(b: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _check(_lib.su2_batch_polyakov(b, _host_ptr(out)), "su2_batch_polyakov")
    return out


def su2_batch_get_links(b: int, i: int, ns: int, nt: int) -> np.ndarray:
    out = np.empty((ns ** 3 * nt, 4, 4), dtype=np.float32)
    _check(_lib.su2_batch_get_links(b, i, _host_ptr(out)), "su2_batch_get_links")
    return out


def su2_batch_set_config(b: int, queue_depth: int, grid: int = 0) -> None:
    _check(_lib.su2_batch_set_config(b, queue_depth, grid), "su2_batch_set_config")


def su2_batch_set_launch(b: int, queue_depth: int, threads: int, grid: int = 0) -> None:
    _check(_lib.su2_batch_set_launch(b, queue_depth, threads, grid), "su2_batch_set_launch")


def su2_batch_set_sampler(b: int, sampler: int) -> None:
    _check(_lib.su2_batch_set_sampler(b, int(sampler)), "su2_batch_set_sampler")


def su2_batch_launch_info(b: int):
    """(queue depth, threads per block, grid) of the current launch."""
    r, t, g = _i32(), _i32(), _i32()
    _check(_lib.su2_batch_launch_info(b, ctypes.byref(r), ctypes.byref(t), ctypes.byref(g)), "su2_batch_launch_info")
    return r.value, t.value, g.value


def su2_batch_autotune(b: int, sweeps: int = 3):
    r, g = _i32(), _i32()
    _check(_lib.su2_batch_autotune(b, sweeps, ctypes.byref(r), ctypes.byref(g)), "su2_batch_autotune")
    return r.value, g.value


def su2_batch_info(b: int) -> dict:
    n, sw, r, g, gr = _i32(), _u32(), _i32(), _i32(), _i32()
    _check(_lib.su2_batch_info(b, ctypes.byref(n), ctypes.byref(sw), ctypes.byref(r), ctypes.byref(g),
                               ctypes.byref(gr)), "su2_batch_info")
    return {"n": n.value, "sweep": sw.value, "queue_depth": r.value, "grid": g.value, "graphs": bool(gr.value)}


def su2_selftest_barrier_timeout(blocks: int, timeout_ns: int) -> int:
    out = _u32()
    _check(_lib.su2_selftest_barrier_timeout(blocks, timeout_ns, ctypes.byref(out)), "su2_selftest_barrier_timeout")
    return out.value


def su2_selftest_mbar_timeout(blocks: int, polls: int) -> int:
    out = _u32()
    _check(_lib.su2_selftest_mbar_timeout(blocks, polls, ctypes.byref(out)), "su2_selftest_mbar_timeout")
    return out.value


def su2_selftest_mma(a_bf16: np.ndarray, b_bf16: np.ndarray) -> np.ndarray:
    """D = A B^T on the tensor cores; A (128, K) and B (32, K) as uint16 BF16 bits."""
    a = np.ascontiguousarray(a_bf16, dtype=np.uint16)
    b = np.ascontiguousarray(b_bf16, dtype=np.uint16)
    k = a.shape[1]
    d = np.zeros((128, 32), dtype=np.float32)
    _check(_lib.su2_selftest_mma(_host_ptr(a), _host_ptr(b), k, _host_ptr(d)), "su2_selftest_mma")
    return d


def su2_status_str(status: int) -> str:
    return _lib.su2_status_str(status).decode()


def su2_last_error() -> str:
    return _lib.su2_last_error().decode(errors="replace")


def su2_abi_version() -> int:
    return _lib.su2_abi_version()
