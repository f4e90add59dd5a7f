"""CPU oracle for pure-gauge lattice SU(2) (Cardoso & Bicudo, LAT2010).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check of the entry module and
the CPU-baseline leg of the benchmark are the only users; the CUDA library never
imports, links or calls anything here, and this package never touches it.

The arithmetic lives in plain C (``su2_oracle.c``, ``su2_oracle_learned.c``);
this module builds it with gcc and exposes numpy-friendly wrappers.  Links are
stored in the natural layout ``links[site, mu, c]`` with sites in lexicographic
order ``((t*Ns + z)*Ns + y)*Ns + x`` and ``c`` = a0..a3 (Sec. 2 quaternions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["su2_oracle.c", "su2_oracle_learned.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Flags that keep binary32 arithmetic exactly as written: no contraction of
# a*b+c into fma (gcc contracts by default on aarch64), no fast-math.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``liboracle.so`` (OpenMP if gcc supports it)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    for extra in (["-fopenmp"], []):
        cmd = ["gcc", *CFLAGS, *extra, *srcs, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB_PATH)
            return _LIB_PATH
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u32, u64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        f32, f64 = ctypes.c_float, ctypes.c_double
        sig = {
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_u01": (f32, [u32]),
            "orc_u01_log": (f32, [u32]),
            "orc_logf": (f32, [f32]),
            "orc_expf": (f32, [f32]),
            "orc_logf_v": (None, [P, P, i64]),
            "orc_expf_v": (None, [P, P, i64]),
            "orc_sincos2pi_v": (None, [P, P, P, i64]),
            "orc_quat_mul": (None, [P, P, P]),
            "orc_cold_start": (None, [i32, i32, P]),
            "orc_hot_start": (i32, [i32, i32, u64, P]),
            "orc_staple": (None, [i32, i32, P, i64, i32, P]),
            "orc_heatbath_link": (i32, [f32, P, u64, u32, u32, i32, i32, P]),
            "orc_creutz_a0": (f32, [f32, u64, u32, u32, i32, i32, ctypes.POINTER(i32)]),
            "orc_heatbath_phase": (i64, [i32, i32, f64, u64, u32, i32, i32, P, ctypes.POINTER(i64), i32]),
            "orc_heatbath_sweep": (i64, [i32, i32, f64, u64, u32, P, P, i32]),
            "orc_site_plaquette": (f32, [i32, i32, P, i64]),
            "orc_site_plaquettes": (None, [i32, i32, P, P]),
            "orc_plaquette": (f64, [i32, i32, P]),
            "orc_plaquette_f64": (f64, [i32, i32, P]),
            "orc_site_polyakov": (f32, [i32, i32, P, i64]),
            "orc_polyakov": (f64, [i32, i32, P]),
            "orc_polyakov_f64": (f64, [i32, i32, P]),
            "orc_reunitarize": (None, [i32, i32, P]),
            "orc_max_threads": (i32, []),
            "orc_creutz_a0_v": (None, [f32, u64, u32, u32, i64, P, P]),
            "orc_creutz_x_a0_v": (None, [P, P, i64, P, P]),
            "orc_heatbath_link_v": (None, [f32, P, u64, u32, u32, i32, i32, i64, P, P]),
            "orc_heatbath_sweep_kp": (i64, [i32, i32, f64, u64, u32, P, P, i32]),
            "orc_heatbath_phase_kp": (i64, [i32, i32, f64, u64, u32, i32, i32, P, ctypes.POINTER(i64), i32]),
            "orc_kp_a0_v": (None, [f32, u64, u32, i64, P, P]),
            "orc_slab_phase": (i64, [i32, i32, i32, i32, f64, u64, u32, i32, i32, i32, P, ctypes.POINTER(i64), i32]),
            "orc_overrelax_link": (None, [P, P]),
            "orc_wilson_loop_at": (f32, [i32, i32, P, i64, i32, i32, i32]),
            "orc_wilson_loops": (None, [i32, i32, P, i32, i32, P, i32]),
            "orc_overrelax_phase": (None, [i32, i32, i32, i32, P, i32]),
            "orc_overrelax_sweep": (None, [i32, i32, P, i32]),
            "orc_mlp_forward": (None, [P, f32, P]),
            "orc_spline_params": (None, [P, P]),
            "orc_spline_forward": (f32, [P, f32, P]),
            "orc_spline_inverse": (f32, [P, f32, P]),
            "orc_spline_forward_v": (None, [P, P, P, P, i64]),
            "orc_spline_inverse_v": (None, [P, P, P, P, i64]),
            "orc_proposal_table": (None, [P, f32, f32, i32, P]),
            "orc_table_params": (None, [P, i32, f32, f32, f32, P]),
            "orc_learned_link": (i32, [P, i32, f32, f32, f32, f32, f32, P, P, u64, u32, u32, i32, i32, P]),
            "orc_learned_phase": (i64, [i32, i32, f64, u64, u32, i32, i32, P, P, i32, f32, f32, f32, f32]),
            "orc_learned_sweep": (i64, [i32, i32, f64, u64, u32, P, P, i32, f32, f32, f32, f32, P]),
            "orc_learned_chain": (i64, [P, i32, f32, f32, f32, f32, f32, P, P, u64, i64, P]),
            "orc_learned_link_net": (i32, [P, f32, P, P, u64, u32, u32, i32, i32, P]),
            "orc_learned_sweep_net": (i64, [i32, i32, f64, u64, u32, P, P, P]),
            "orc_learned_chain_net": (i64, [P, f32, P, P, u64, i64, P]),
            "orc_collect_pairs": (i64, [i32, i32, f64, u64, u32, i32, i32, i32, P, P]),
            "orc_nll_grad": (f64, [P, P, i64, P]),
            "orc_nll_outputs": (f64, [P, f64, P]),
            "orc_spline_d": (None, [P, f64, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def volume(ns: int, nt: int) -> int:
    return ns * ns * ns * nt


def new_links(ns: int, nt: int) -> np.ndarray:
    return np.zeros((volume(ns, nt), 4, 4), dtype=np.float32)


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(x: int) -> float:
    return _load().orc_u01(x)


def u01_log(x: int) -> float:
    """The uniform in [2^-33, 1] that feeds a logarithm (Creutz's x, the
    Kennedy-Pendleton exponentials)."""
    return _load().orc_u01_log(x)


def logf(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    _load().orc_logf_v(_ptr(x), _ptr(y), x.size)
    return y


def expf(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    _load().orc_expf_v(_ptr(x), _ptr(y), x.size)
    return y


def sincos2pi(u):
    u = np.ascontiguousarray(u, dtype=np.float32)
    s = np.empty_like(u)
    c = np.empty_like(u)
    _load().orc_sincos2pi_v(_ptr(u), _ptr(s), _ptr(c), u.size)
    return s, c


def quat_mul(a, b) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    c = np.zeros(4, dtype=np.float32)
    _load().orc_quat_mul(_ptr(a), _ptr(b), _ptr(c))
    return c


# ------------------------------------------------------------------- lattice
def cold_start(ns: int, nt: int) -> np.ndarray:
    links = new_links(ns, nt)
    _load().orc_cold_start(ns, nt, _ptr(links))
    return links


def hot_start(ns: int, nt: int, seed: int) -> np.ndarray:
    links = new_links(ns, nt)
    err = _load().orc_hot_start(ns, nt, seed, _ptr(links))
    if err:
        raise RuntimeError(f"hot start: {err} links without two disk points")
    return links


def staple(ns: int, nt: int, links: np.ndarray, site: int, mu: int) -> np.ndarray:
    v = np.zeros(4, dtype=np.float32)
    _load().orc_staple(ns, nt, _ptr(links), site, mu, _ptr(v))
    return v


def heatbath_link(beta: float, v, seed: int, eo: int, sweep: int, parity: int, mu: int):
    """Returns (new link, trials); trials = -1 if the trial cap was hit."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    out = np.zeros(4, dtype=np.float32)
    n = _load().orc_heatbath_link(beta, _ptr(v), seed, eo, sweep, parity, mu, _ptr(out))
    return out, n


def creutz_a0(bk: float, seed: int, eo: int, sweep: int = 0, parity: int = 0, mu: int = 0):
    t = ctypes.c_int(0)
    a0 = _load().orc_creutz_a0(bk, seed, eo, sweep, parity, mu, ctypes.byref(t))
    return a0, t.value


def creutz_a0_many(bk: float, seed: int, n: int, eo0: int = 0, sweep: int = 0):
    """n draws of a0 at fixed beta*k (draw i uses even/odd index eo0 + i)."""
    a0 = np.zeros(n, dtype=np.float32)
    t = np.zeros(n, dtype=np.int32)
    _load().orc_creutz_a0_v(bk, seed, eo0, sweep, n, _ptr(a0), _ptr(t))
    return a0, t


def creutz_x_a0(bk, w):
    """Single Creutz trials: for beta k = bk[i] and first Philox word w[i],
    x = e + r1 (1 - e) and the candidate a0 (clamped), as the heat-bath link
    forms them."""
    bk = np.ascontiguousarray(bk, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    assert bk.shape == w.shape
    x = np.empty_like(bk)
    a0 = np.empty_like(bk)
    _load().orc_creutz_x_a0_v(_ptr(bk), _ptr(w), bk.size, _ptr(x), _ptr(a0))
    return x, a0


def heatbath_link_many(beta: float, v, seed: int, eo: int, parity: int, mu: int, n: int, sweep0: int = 0):
    """n independent heat-bath updates of one link with staple v (sweep numbers
    sweep0 .. sweep0+n-1).  Returns (links[n,4], trials[n])."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    out = np.zeros((n, 4), dtype=np.float32)
    t = np.zeros(n, dtype=np.int32)
    _load().orc_heatbath_link_v(beta, _ptr(v), seed, eo, sweep0, parity, mu, n, _ptr(out), _ptr(t))
    return out, t


def heatbath_sweep(ns: int, nt: int, beta: float, seed: int, sweep: int, links: np.ndarray,
                   nthreads: int = 1) -> np.ndarray:
    """One sweep in place; returns the trial count of each of the 8 phases
    (index 2*mu + parity).  Raises if a sampler hit its trial cap."""
    trials = np.zeros(8, dtype=np.int64)
    err = _load().orc_heatbath_sweep(ns, nt, beta, seed, sweep, _ptr(links), _ptr(trials), nthreads)
    if err:
        raise RuntimeError(f"{err} links hit the trial cap")
    return trials


def slab_phase(ns: int, nt: int, t0: int, nt_local: int, beta: float, seed: int, sweep: int, mu: int,
               parity: int, slab: np.ndarray, kp: bool = False, nthreads: int = 1) -> int:
    """One phase on a time slab in place (slab: Ns^3 x (nt_local + 2) sites,
    ghosts at local slices 0 and nt_local + 1); returns its trial count."""
    assert slab.shape == (ns ** 3 * (nt_local + 2), 4, 4) and slab.dtype == np.float32
    t = ctypes.c_int64(0)
    err = _load().orc_slab_phase(ns, nt, t0, nt_local, beta, seed, sweep, mu, parity, int(kp), _ptr(slab),
                                 ctypes.byref(t), nthreads)
    if err:
        raise RuntimeError(f"{err} links hit the trial cap")
    return t.value


def heatbath_phase_kp(ns: int, nt: int, beta: float, seed: int, sweep: int, mu: int, parity: int,
                      links: np.ndarray, nthreads: int = 1) -> int:
    """One Kennedy-Pendleton phase in place; returns its trial count."""
    t = ctypes.c_int64(0)
    err = _load().orc_heatbath_phase_kp(ns, nt, beta, seed, sweep, mu, parity, _ptr(links), ctypes.byref(t),
                                        nthreads)
    if err:
        raise RuntimeError(f"{err} links hit the trial cap")
    return t.value


def heatbath_sweep_kp(ns: int, nt: int, beta: float, seed: int, sweep: int, links: np.ndarray,
                      nthreads: int = 1) -> np.ndarray:
    """One sweep with the Kennedy-Pendleton sampler (Creutz below beta k = 2)."""
    trials = np.zeros(8, dtype=np.int64)
    err = _load().orc_heatbath_sweep_kp(ns, nt, beta, seed, sweep, _ptr(links), _ptr(trials), nthreads)
    if err:
        raise RuntimeError(f"{err} links hit the trial cap")
    return trials


def overrelax_link(v, u) -> np.ndarray:
    """U' = U~^dag U^dag U~^dag for staple v (the reflection that keeps Tr UV)."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    out = np.array(u, dtype=np.float32, copy=True)
    _load().orc_overrelax_link(_ptr(v), _ptr(out))
    return out


def overrelax_phase(ns: int, nt: int, mu: int, parity: int, links: np.ndarray, nthreads: int = 1) -> None:
    _load().orc_overrelax_phase(ns, nt, mu, parity, _ptr(links), nthreads)


def overrelax_sweep(ns: int, nt: int, links: np.ndarray, nthreads: int = 1) -> None:
    """One over-relaxation sweep (mu = 0..3, even then odd), in place."""
    _load().orc_overrelax_sweep(ns, nt, _ptr(links), nthreads)


def wilson_loops(ns: int, nt: int, links: np.ndarray, rmax: int, tmax: int, nthreads: int = 1) -> np.ndarray:
    """W[R-1, T-1]: mean (1/2) Tr of the R x T space-time loops (binary32 per
    loop, binary64 mean over sites and the three spatial directions)."""
    out = np.zeros(rmax * tmax, dtype=np.float64)
    _load().orc_wilson_loops(ns, nt, _ptr(links), rmax, tmax, _ptr(out), nthreads)
    return out.reshape(rmax, tmax)


def wilson_loop_at(ns: int, nt: int, links: np.ndarray, site: int, i: int, R: int, T: int) -> float:
    return float(_load().orc_wilson_loop_at(ns, nt, _ptr(links), site, i, R, T))


def kp_a0_many(bk: float, seed: int, n: int, eo0: int = 0):
    a0 = np.zeros(n, dtype=np.float32)
    t = np.zeros(n, dtype=np.int32)
    _load().orc_kp_a0_v(bk, seed, eo0, n, _ptr(a0), _ptr(t))
    return a0, t


def heatbath_phase(ns: int, nt: int, beta: float, seed: int, sweep: int, mu: int, parity: int,
                   links: np.ndarray, nthreads: int = 1) -> int:
    t = ctypes.c_int64(0)
    err = _load().orc_heatbath_phase(ns, nt, beta, seed, sweep, mu, parity, _ptr(links), ctypes.byref(t), nthreads)
    if err:
        raise RuntimeError(f"{err} links hit the trial cap")
    return t.value


def plaquette(ns: int, nt: int, links: np.ndarray) -> float:
    return _load().orc_plaquette(ns, nt, _ptr(links))


def plaquette_f64(ns: int, nt: int, links: np.ndarray) -> float:
    return _load().orc_plaquette_f64(ns, nt, _ptr(links))


def site_plaquettes(ns: int, nt: int, links: np.ndarray) -> np.ndarray:
    out = np.zeros(volume(ns, nt), dtype=np.float32)
    _load().orc_site_plaquettes(ns, nt, _ptr(links), _ptr(out))
    return out


def polyakov(ns: int, nt: int, links: np.ndarray) -> float:
    return _load().orc_polyakov(ns, nt, _ptr(links))


def polyakov_f64(ns: int, nt: int, links: np.ndarray) -> float:
    return _load().orc_polyakov_f64(ns, nt, _ptr(links))


def reunitarize(ns: int, nt: int, links: np.ndarray) -> None:
    _load().orc_reunitarize(ns, nt, _ptr(links))


def max_threads() -> int:
    return _load().orc_max_threads()


# ------------------------------------------------------- learned proposal
N_WEIGHTS = 1947      # 1945 trainable + input mean and scale
N_TRAIN = 1945
N_PARAMS = 27         # spline knots x0..x8, y0..y8, derivatives d0..d8


def mlp_forward(w, s: float) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float32)
    o = np.zeros(25, dtype=np.float32)
    _load().orc_mlp_forward(_ptr(w), s, _ptr(o))
    return o


def spline_params(o) -> np.ndarray:
    o = np.ascontiguousarray(o, dtype=np.float32)
    p = np.zeros(N_PARAMS, dtype=np.float32)
    _load().orc_spline_params(_ptr(o), _ptr(p))
    return p


def spline_forward(p, z):
    p = np.ascontiguousarray(p, dtype=np.float32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    a, fp = np.empty_like(z), np.empty_like(z)
    _load().orc_spline_forward_v(_ptr(p), _ptr(z), _ptr(a), _ptr(fp), z.size)
    return a, fp


def spline_inverse(p, a):
    p = np.ascontiguousarray(p, dtype=np.float32)
    a = np.ascontiguousarray(a, dtype=np.float32)
    z, fp = np.empty_like(a), np.empty_like(a)
    _load().orc_spline_inverse_v(_ptr(p), _ptr(a), _ptr(z), _ptr(fp), a.size)
    return z, fp


def proposal_table(w, s_lo: float, s_hi: float, G: int = 256) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float32)
    t = np.zeros((G, N_PARAMS), dtype=np.float32)
    _load().orc_proposal_table(_ptr(w), s_lo, s_hi, G, _ptr(t))
    return t


def table_params(table, s_lo, s_hi, s) -> np.ndarray:
    table = np.ascontiguousarray(table, dtype=np.float32)
    p = np.zeros(N_PARAMS, dtype=np.float32)
    _load().orc_table_params(_ptr(table), table.shape[0], s_lo, s_hi, s, _ptr(p))
    return p


def learned_sweep(ns, nt, beta, seed, sweep, links, table, s_lo, s_hi, mean, scale) -> np.ndarray:
    table = np.ascontiguousarray(table, dtype=np.float32)
    acc = np.zeros(8, dtype=np.int64)
    _load().orc_learned_sweep(ns, nt, beta, seed, sweep, _ptr(links), _ptr(table), table.shape[0], s_lo, s_hi, mean,
                              scale, _ptr(acc))
    return acc


def learned_chain(table, s_lo, s_hi, mean, scale, beta, v, old0, seed, n):
    table = np.ascontiguousarray(table, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    old0 = np.ascontiguousarray(old0, dtype=np.float32)
    a0 = np.zeros(n, dtype=np.float32)
    acc = _load().orc_learned_chain(_ptr(table), table.shape[0], s_lo, s_hi, mean, scale, beta, _ptr(v), _ptr(old0),
                                    seed, n, _ptr(a0))
    return a0, acc


def learned_sweep_net(ns, nt, beta, seed, sweep, links, w) -> np.ndarray:
    """One learned sweep in place with the network evaluated at every link's
    beta k (the proposal as defined, no table); accepted links per phase."""
    w = np.ascontiguousarray(w, dtype=np.float32)
    assert w.size == N_WEIGHTS
    acc = np.zeros(8, dtype=np.int64)
    _load().orc_learned_sweep_net(ns, nt, beta, seed, sweep, _ptr(links), _ptr(w), _ptr(acc))
    return acc


def learned_chain_net(w, beta, v, old0, seed, n):
    w = np.ascontiguousarray(w, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    old0 = np.ascontiguousarray(old0, dtype=np.float32)
    a0 = np.zeros(n, dtype=np.float32)
    acc = _load().orc_learned_chain_net(_ptr(w), beta, _ptr(v), _ptr(old0), seed, n, _ptr(a0))
    return a0, acc


def collect_pairs(ns, nt, beta, seed, sweep, mu, parity, stride, links) -> np.ndarray:
    n_max = ns ** 3 * nt // 2 // stride + 1
    pairs = np.zeros((n_max, 2), dtype=np.float32)
    n = _load().orc_collect_pairs(ns, nt, beta, seed, sweep, mu, parity, stride, _ptr(links), _ptr(pairs))
    return pairs[:n]


def nll_grad(w, pairs, want_grad=True):
    """binary64 mean -log q(a0 | beta k) and its gradient (1945 weights)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    pairs = np.ascontiguousarray(pairs, dtype=np.float32)
    g = np.zeros(N_TRAIN, dtype=np.float64) if want_grad else None
    v = _load().orc_nll_grad(_ptr(w), _ptr(pairs), pairs.shape[0], _ptr(g) if want_grad else None)
    return v, g


def nll_outputs(o, a, want_grad=True):
    o = np.ascontiguousarray(o, dtype=np.float64)
    g = np.zeros(25, dtype=np.float64) if want_grad else None
    v = _load().orc_nll_outputs(_ptr(o), a, _ptr(g) if want_grad else None)
    return v, g


def spline_d(o, z):
    o = np.ascontiguousarray(o, dtype=np.float64)
    a, fp, zi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().orc_spline_d(_ptr(o), z, ctypes.byref(a), ctypes.byref(fp), ctypes.byref(zi))
    return a.value, fp.value, zi.value
