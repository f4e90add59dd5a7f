#!/usr/bin/env python3
"""Benchmark of the SU(2) checkerboard heat bath on GB300.

Workload (the paper's benchmark shape, Sec. 4.1 and the 48^4 figure of the
abstract): a 48^4 lattice at beta = 6.0 from a hot start (Philox seed 3, plus
the rank on N > 1 GPUs), links as binary32 quaternions.  One step = one
heat-bath sweep (8 even/odd phases) + the plaquette + the Polyakov loop.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` = link updates/s over all ranks,
device-timed with CUDA events around K steps with the links resident in HBM
(340 MB, larger than the 129 MB L2, so no flush is needed).  `e2e` = the same
metric through the C ABI with host buffers (configuration in from pinned host
memory, sweep, observables, configuration out), copies inside the timed
region.  `roofline` = algorithmic bytes of the heat-bath phase kernel over its
duration: CUDA events on the launching stream around K unmeasured sweeps
replayed back to back, over their 8 K phase launches (the per-launch
event-bracketed duration is reported beside it).
`--impl reference` times the CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NS = NT = 48
BETA = 6.0
SEED = 3
VOL = NS ** 3 * NT
LINKS = 4 * VOL
METRIC = "SU(2) heat-bath link updates/s (plain vs learned, τ_int-adj.) & % of HBM peak"
UNIT = "link updates/s"
# 10^6 configurations of 48^4 per day on two GTX 295 cards (one sweep each)
PAPER_RATE = 1.0e6 * LINKS / 86400.0
BYTES_PER_UPDATE = 128  # reads 3.5 V + writes 0.5 V float4 per phase of V/2 updates
BYTES_PER_LEARNED_UPDATE = 144  # + the old link of the updated direction and parity
BYTES_PER_OR_UPDATE = 144  # over-relaxation: the staple links, the old link, the new link
N_OR = 3  # over-relaxation sweeps after each heat-bath sweep in the compound form
TRAIN_BATCH = 16384  # training mini-batch of the learned proposal
# the phase kernel of each plain sampler: its source files (for the source
# digest that ties a committed ncu summary to the current kernel) and summary
SAMPLERS = {
    "kp": {"kernel": "kp_phase_kernel", "name": "Kennedy-Pendleton",
           "sources": ["paper_1010_1486_gb300/csrc/kp.cu", "paper_1010_1486_gb300/csrc/kp_device.cuh",
                       "paper_1010_1486_gb300/csrc/su2_device.cuh", "paper_1010_1486_gb300/csrc/staple.cuh"],
           "profile": os.path.join(ROOT, "profiles", "kp_phase_48x48x48x48_beta6.md")},
    "creutz": {"kernel": "hb_phase_kernel", "name": "Creutz",
               "sources": ["paper_1010_1486_gb300/csrc/heatbath.cu", "paper_1010_1486_gb300/csrc/su2_device.cuh",
                           "paper_1010_1486_gb300/csrc/staple.cuh", "paper_1010_1486_gb300/csrc/creutz_queue.cuh"],
               "profile": os.path.join(ROOT, "profiles", "hb_phase_48x48x48x48_beta6.md")},
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--e2e-in-flight", type=int, default=4, help="configurations in flight in the e2e pipeline")
    ap.add_argument("--tau-sweeps", type=int, default=8000,
                    help="sweeps per form for tau_int and the plaquette comparison (0 = skip)")
    ap.add_argument("--therm", type=int, default=1500, help="thermalisation sweeps before the form comparison")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--learned-pairs", type=int, default=1_000_000, help="training pairs (0 = skip the learned form)")
    ap.add_argument("--train-steps", type=int, default=3000, help="Adam steps of each of the two training stages")
    ap.add_argument("--batched-steps", type=int, default=200, help="sweeps of the 64-lattice batch (0 = skip)")
    ap.add_argument("--sampler", choices=sorted(SAMPLERS), default="kp",
                    help="a0 sampler of the headline plain heat bath (both are exact; kp = Kennedy-Pendleton)")
    ap.add_argument("--small", type=int, default=1, help="time the small, L2-resident workloads too (0 = skip)")
    ap.add_argument("--slabs", type=int, default=20,
                    help="sweeps of the 48^4 lattice split into two time slabs on this GPU (0 = skip)")
    return ap.parse_args(argv)


# ------------------------------------------------------------- distributed
class Dist:
    def __init__(self, want: int):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        if want > 1 and self.world != want:
            raise SystemExit(f"--gpus {want} needs torchrun with {want} processes (WORLD_SIZE={self.world})")
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist

            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def reduce(self, value: float, op: str) -> float:
        """max or sum of a float over ranks (gloo on CPU or nccl on GPU)."""
        if not self.pg:
            return value
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------ clocks
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index: int, path: str):
        self.gpu_index, self.path, self.proc = gpu_index, path, None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu_index), "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append({"sm": float(f[1]), "max": float(f[2]), "power": float(f[3]),
                             "reasons": [r for r, v in zip(REASONS, f[5:9]) if v.lower() == "active"]})
            except ValueError:
                continue
        if not rows:
            return None
        load = [r for r in rows if r["power"] > 200.0] or rows
        reasons = sorted({x for r in load for x in r["reasons"]})
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": reasons, "samples": len(load), "power_w_max": max(r["power"] for r in rows)}


class NvmlClockSampler:
    """SM clock, power and clock-event reasons read through NVML (read only:
    nvmlDeviceGetClockInfo, GetMaxClockInfo, GetPowerUsage and the current
    clock-event reasons) every 2 ms on a thread while the timed work runs, so
    that every sample falls inside the timed region."""

    SM = 1  # NVML_CLOCK_SM
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, uuid: str | None, index: int):
        import ctypes
        import threading

        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit_v2 failed")
        self.h = ctypes.c_void_p()
        rc = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) if uuid else 1
        if rc != 0:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h))
        if rc != 0:
            self.lib.nvmlShutdown()
            raise OSError("no NVML handle for the device")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.rows = []
        self.done = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _sample(self):
        c = self.ct
        mhz, mx, mw, rs = c.c_uint(), c.c_uint(), c.c_uint(), c.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, c.byref(mhz)) != 0:
            return
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, c.byref(mx))
        self.lib.nvmlDeviceGetPowerUsage(self.h, c.byref(mw))
        self.reasons_fn(self.h, c.byref(rs))
        self.rows.append({"sm": float(mhz.value), "max": float(mx.value), "power": mw.value / 1000.0,
                          "reasons": [r for r, b in self.BITS.items() if rs.value & b]})

    def _run(self):
        while not self.done.is_set():
            self._sample()
            time.sleep(0.002)

    def start(self):
        self.thread.start()

    def stop(self):
        self.done.set()
        self.thread.join()
        self.lib.nvmlShutdown()
        rows = self.rows
        if not rows:
            return None
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": sorted({x for r in rows for x in r["reasons"]}), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows), "source": "NVML, every 2 ms inside the timed region"}


def clock_sampler(torch, local_rank: int, gpu_index: int, rank: int):
    """The NVML sampler for the device, else nvidia-smi in a subprocess."""
    try:
        uuid = getattr(torch.cuda.get_device_properties(local_rank), "uuid", None)
        uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else (str(uuid) if uuid else None)
        return NvmlClockSampler(uuid, gpu_index)
    except (OSError, AttributeError):
        return ClockSampler(gpu_index, os.path.join(tempfile.gettempdir(), f"su2_clocks_rank{rank}.csv"))


# ------------------------------------------------------- measured peaks etc
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_digest(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic_per_launch(sampler: str):
    """DRAM bytes per phase launch from the committed ncu summary of that
    sampler's kernel, if it was taken on the current source; else None."""
    spec = SAMPLERS[sampler]
    if not os.path.exists(spec["profile"]):
        return None
    text = open(spec["profile"]).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != source_digest(spec["sources"]):
        return None
    return float(m.group(1))


# ---------------------------------------------------------------- our arm
def run_ours(args, dist):
    import numpy as np
    import torch

    from paper_1010_1486_gb300 import su2
    from paper_1010_1486_gb300.analysis import tau_int

    torch.cuda.set_device(dist.local_rank)
    su2.use_torch_allocator()
    stream = torch.cuda.Stream()
    seed = SEED + dist.rank
    sampler = su2.SU2_SAMPLER_KP if args.sampler == "kp" else su2.SU2_SAMPLER_CREUTZ
    lat = su2.su2_create(NS, NT, BETA, seed, su2.SU2_HOT, stream=stream)
    try:
        su2.su2_set_sampler(lat, sampler)
        su2.su2_generate(lat, args.warmup, 1, 0)  # also captures the sweep's CUDA graph
        gpu_index = dist.local_rank
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            try:
                gpu_index = int(vis.split(",")[dist.local_rank])
            except ValueError:
                pass
        clocks = clock_sampler(torch, dist.local_rank, gpu_index, dist.rank)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        # the timed steps: one counter reset, then each sweep with its
        # measurement replayed from the lattice's CUDA graph (10 kernels: 8
        # phases, the Polyakov loop with the plaquette's slot sum, the
        # counter advance)
        ev0.record(stream)
        plaq, poly, st = su2.su2_generate(lat, args.steps, 1, 0)
        ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        dist.barrier()
        ms = ev0.elapsed_time(ev1)
        # the phase kernel's duration, for the roofline: the same number of
        # sweeps without the measurement, replayed back to back from the
        # graph (8 phase launches + the counter advance per sweep), CUDA
        # events around them on the lattice's stream, over 8 launches a sweep
        phase_s, phase_s_events = phase_kernel_time(su2, lat, torch, stream, args.steps)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms_max = dist.reduce(ms, "max")
        updates = dist.reduce(float(st["link_updates"]), "sum")
        value = updates / (ms_max * 1e-3)
        peak, peak_kind = measured_peaks()
        achieved = BYTES_PER_UPDATE * (VOL // 2) / phase_s / 1e9
        trials_per_update = sum(st["trials"]) / st["link_updates"]
        traffic = ncu_traffic_per_launch(args.sampler)

        # end to end through the C ABI with host buffers
        e2e = None
        if args.e2e_steps > 0:
            e2e = run_e2e(args, dist, lat, su2, torch)

        forms = None
        if args.learned_pairs > 0:
            forms = compare_forms(args, dist, lat, su2, torch, stream, tau_int)
    finally:
        su2.su2_destroy(lat)

    batched = None
    if args.batched_steps > 0:
        batched = run_batched(args, dist, su2, torch)
    small = run_small(args, dist, su2, torch) if args.small else None
    slabs = run_slabs(args, dist, su2, torch, 8 * phase_s) if args.slabs > 0 else None

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_RATE, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{NS}^4 lattice, beta={BETA}, hot start (Philox seed {SEED}+rank), one step = "
                               "heat-bath sweep (8 even/odd phases) + plaquette + Polyakov loop",
                   "lattice": [NS, NS, NS, NT], "beta": BETA, "start": "hot",
                   "form": f"plain heat bath ({SAMPLERS[args.sampler]['name']} a0 sampler)",
                   "parallelism": "independent replicas" if dist.world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (340 MB of links vs 129 MB L2), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": SAMPLERS[args.sampler]["kernel"],
                     # ncu's DRAM bytes of one launch over the live launch duration
                     "traffic_gbs": traffic / phase_s / 1e9 if traffic else None,
                     "peak_source": f"{peak_kind} hbm_gbs", "bytes_per_launch": BYTES_PER_UPDATE * (VOL // 2),
                     "avg_launch_us": phase_s * 1e6, "timing": PHASE_TIMING,
                     "event_bracketed_launch_us": phase_s_events * 1e6},
        "without_measurement": {
            "value": dist.reduce(float(LINKS), "sum") / (8 * phase_s), "unit": UNIT,
            "ms_per_sweep": 8 * phase_s * 1e3, "sweeps_per_s": 1.0 / (8 * phase_s),
            "how": "the roofline pass: unmeasured sweeps replayed back to back (8 phases + the counter advance)"},
        "e2e": e2e,
        "gpu_launches": 10 * args.steps + 1,  # + the counter reset before the replays
        "clocks": clk,
        "trials_per_update": trials_per_update,
        "plaquette_last": float(plaq[-1]), "polyakov_last": float(poly[-1]),
        "forms": forms,
        "batched": batched,
        "small_workloads": small,
        "time_slabs": slabs,
    }
    if forms and "value_tau_adjusted" in forms:
        result["value_tau_adjusted"] = forms["value_tau_adjusted"]
    return result


PHASE_TIMING = ("back-to-back launches: sweeps without the measurement replayed from the graph, CUDA events around "
                "them on the lattice's stream, divided by the 8 phase launches a sweep (the counter-advance kernel "
                "and the gaps count against the phase)")


def phase_kernel_time(su2, lat, torch, stream, steps):
    """Seconds per phase launch, (1) back to back: `steps` unmeasured sweeps
    replayed from the lattice's graph, events around them; (2) with CUDA
    events around every launch (eager launches; includes each launch's
    latency)."""
    su2.su2_generate(lat, 2, 0, 0)  # the unmeasured sweep's graph, captured untimed
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    su2.su2_generate(lat, steps, 0, 0)
    e1.record(stream)
    e1.synchronize()
    back_to_back = e0.elapsed_time(e1) * 1e-3 / (8 * steps)
    su2.su2_set_timing(lat, True)
    _, _, st = su2.su2_generate(lat, steps, 0, 0)
    su2.su2_set_timing(lat, False)
    return back_to_back, st["kernel_ms"] / st["kernel_launches"] * 1e-3


def timed(stream, torch, dist, fn):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    out = fn()
    ev1.record(stream)
    ev1.synchronize()
    return dist.reduce(ev0.elapsed_time(ev1), "max"), out


def compare_forms(args, dist, lat, su2, torch, stream, tau_int):
    """The plain heat bath with each exact a0 sampler (Kennedy-Pendleton,
    Creutz), the learned proposal and Kennedy-Pendleton + over-relaxation on
    the same thermalised 48^4 lattice.

    1. Thermalisation: `therm` compound sweeps (one Kennedy-Pendleton sweep +
       N_OR over-relaxation sweeps; over-relaxation moves the slow, long-
       wavelength modes that a heat bath alone relaxes diffusively).
    2. (beta k, a0) pairs from the plain sampler, training on the GPU.
    3. Each form timed over `steps` sweeps (rates and kernel rooflines).
    4. Interleaved blocks per round: Kennedy-Pendleton (the reference),
       learned, Creutz, Kennedy-Pendleton + over-relaxation; a final
       reference block.  Each sweep records the plaquette and the Polyakov
       loop.  tau_int per form for the plaquette and for |L| (a slow
       observable), the blocks of a form pooled as replicas about their common
       mean; the drift of the reference blocks against their scatter; each
       form's plaquette against the reference interpolated at its blocks'
       centres (analysis.interleaved_offset)."""
    from paper_1010_1486_gb300 import learn
    from paper_1010_1486_gb300.analysis import block_drift, interleaved_offset

    import numpy as np

    KP, CR = su2.SU2_SAMPLER_KP, su2.SU2_SAMPLER_CREUTZ
    su2.su2_set_sampler(lat, KP)
    su2.su2_set_overrelax(lat, N_OR)
    su2.su2_generate(lat, args.therm, 0, 0)
    su2.su2_set_overrelax(lat, 0)
    t0 = time.perf_counter()
    pairs = learn.collect(lat, NS, NT, args.learned_pairs, sweeps_between=1)
    t1 = time.perf_counter()
    w, losses, s_lo, s_hi = learn.train(pairs, steps=args.train_steps, batch=TRAIN_BATCH, lr=3e-3, seed=11,
                                        tail_steps=args.train_steps, tail_lr=3e-4)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del pairs
    su2.su2_set_proposal(lat, w, s_lo, s_hi, 256)
    peak, _ = measured_peaks()

    def roof(kernel, phase_s, nbytes, timing, events_s=None):
        a = nbytes * (VOL // 2) / phase_s / 1e9
        r = {"bound": "hbm", "kernel": kernel, "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
             "avg_launch_us": phase_s * 1e6, "bytes_per_launch": nbytes * (VOL // 2), "timing": timing}
        if events_s is not None:
            r["event_bracketed_launch_us"] = events_s * 1e6
        return r

    out = {"lattice": f"thermalised 48^4, beta = 6.0 (after {args.therm} compound sweeps of Kennedy-Pendleton + "
                      f"{N_OR} over-relaxation)"}
    sweep_s = {}
    for key, sampler, kernel in (("kennedy_pendleton", KP, "kp_phase_kernel"), ("creutz", CR, "hb_phase_kernel")):
        su2.su2_set_sampler(lat, sampler)
        su2.su2_generate(lat, 2, 1, 0)
        ms, (_, _, st) = timed(stream, torch, dist, lambda: su2.su2_generate(lat, args.steps, 1, 0))
        phase_s, events_s = phase_kernel_time(su2, lat, torch, stream, args.steps)
        sweep_s[key] = 8 * phase_s
        out[key] = {"value": dist.reduce(float(st["link_updates"]), "sum") / (ms * 1e-3), "unit": UNIT,
                    "ms_per_step": ms / args.steps, "trials_per_update": sum(st["trials"]) / st["link_updates"],
                    "roofline": roof(kernel, phase_s, BYTES_PER_UPDATE, PHASE_TIMING, events_s)}
    su2.su2_set_sampler(lat, KP)  # the learned sweeps' fallback sampler
    su2.su2_learned_generate(lat, 2, 1, 0.7)
    ms_l, (_, _, st_l) = timed(stream, torch, dist, lambda: su2.su2_learned_generate(lat, args.steps, 1, 0.7))
    # the learned phase kernel back to back: unmeasured learned sweeps (each
    # also launches the eight gated plain phases, which return at once, and
    # the fallback decision), CUDA events around them, over 8 learned
    # launches a sweep; and with events around every learned launch
    ms_lb, (_, _, st_lb) = timed(stream, torch, dist, lambda: su2.su2_learned_generate(lat, args.steps, 0, 0.7))
    learned_phase_s = ms_lb * 1e-3 / (8 * args.steps)
    su2.su2_set_timing(lat, True)
    _, _, st_lt = su2.su2_learned_generate(lat, args.steps, 1, 0.7)
    su2.su2_set_timing(lat, False)
    learned_events_s = st_lt["kernel_ms"] / max(1, st_lt["kernel_launches"]) * 1e-3
    learned_timing = ("back-to-back launches: unmeasured learned sweeps (with their gated plain phases and the "
                      "fallback decision, which count against the learned phase), CUDA events around them, over "
                      "the 8 learned launches a sweep")
    if st_lb["plain_sweeps"] > 0:  # a fallback sweep ran: keep the per-launch figure
        learned_phase_s = learned_events_s
        learned_timing = "CUDA events around every learned phase launch (each launch's latency included)"
    proposals = st_l["learned_sweeps"] * 4 * VOL
    out["learned"] = {
        "value": dist.reduce(float(st_l["link_updates"]), "sum") / (ms_l * 1e-3), "unit": UNIT,
        "ms_per_step": ms_l / args.steps, "acceptance": sum(st_l["accepted"]) / max(1, proposals),
        "learned_sweeps": st_l["learned_sweeps"], "fallback_sweeps": st_l["plain_sweeps"],
        "fallback_sampler": "Kennedy-Pendleton",
        "roofline": roof("learned_phase_kernel", learned_phase_s, BYTES_PER_LEARNED_UPDATE, learned_timing,
                         learned_events_s),
        "gpu_launches": st_l["kernel_launches"] * 2 + args.steps * 2,
        "training": {"pairs": args.learned_pairs, "steps": 2 * args.train_steps, "batch": TRAIN_BATCH,
                     "schedule": f"{args.train_steps} Adam steps at 3e-3, {args.train_steps} at 3e-4",
                     "collect_s": t1 - t0, "train_s": t2 - t1,
                     "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-50:].mean())}}
    su2.su2_set_overrelax(lat, N_OR)
    su2.su2_generate(lat, 2, 1, 0)
    n_cmp = max(1, args.steps // (N_OR + 1))
    ms_o, (_, _, st_o) = timed(stream, torch, dist, lambda: su2.su2_generate(lat, n_cmp, 1, 0))
    # over-relaxation phase: unmeasured compound sweeps back to back, less the
    # Kennedy-Pendleton sweep timed the same way, over 8 N_OR launches
    su2.su2_generate(lat, 2, 0, 0)
    ms_c, _ = timed(stream, torch, dist, lambda: su2.su2_generate(lat, n_cmp, 0, 0))
    su2.su2_set_timing(lat, True)
    _, _, st_ot = su2.su2_generate(lat, n_cmp, 0, 0)
    su2.su2_set_timing(lat, False)
    su2.su2_set_overrelax(lat, 0)
    or_phase_s = (ms_c * 1e-3 / n_cmp - sweep_s["kennedy_pendleton"]) / (8 * N_OR)
    or_events_s = st_ot["overrelax_ms"] / (8 * st_ot["overrelax_sweeps"]) * 1e-3
    compound_per_s = dist.reduce(float(n_cmp), "sum") / (ms_o * 1e-3)
    out["kp_overrelax"] = {
        "compound_sweep": f"1 Kennedy-Pendleton heat-bath sweep + {N_OR} over-relaxation sweeps",
        "compound_sweeps_per_s": compound_per_s, "ms_per_compound_sweep": ms_o / n_cmp,
        "value": compound_per_s * 4 * VOL * (N_OR + 1), "unit": UNIT + " (heat bath + over-relaxation)",
        "roofline": roof("or_phase_kernel", or_phase_s, BYTES_PER_OR_UPDATE,
                         "back-to-back launches: unmeasured compound sweeps replayed from the graph less the "
                         "Kennedy-Pendleton sweep timed the same way, over the 8 N_OR over-relaxation launches",
                         or_events_s)}
    if args.tau_sweeps <= 0:
        return out

    nblk = 16
    per = max(50, args.tau_sweeps // nblk)
    per_or = max(25, per // (N_OR + 1) * 2)
    blocks = {k: {"P": [], "L": []} for k in ("kennedy_pendleton", "learned", "creutz", "kp_overrelax")}

    def record(key, res):
        blocks[key]["P"].append(np.array(res[0], dtype=np.float64))
        blocks[key]["L"].append(np.abs(np.array(res[1], dtype=np.float64)))

    for k in range(nblk + 1):
        su2.su2_set_sampler(lat, KP)
        record("kennedy_pendleton", su2.su2_generate(lat, per, 1, 0))
        if k == nblk:
            break
        record("learned", su2.su2_learned_generate(lat, per, 1, 0.7))
        su2.su2_set_sampler(lat, CR)
        record("creutz", su2.su2_generate(lat, per, 1, 0))
        su2.su2_set_sampler(lat, KP)
        su2.su2_set_overrelax(lat, N_OR)
        record("kp_overrelax", su2.su2_generate(lat, per_or, 1, 0))
        su2.su2_set_overrelax(lat, 0)
    su2.su2_set_sampler(lat, CR)
    # block centres, as fractions of a round from one reference block's centre
    # to the next (a compound sweep counts as 1 + N_OR sweeps)
    span = 3 * per + (N_OR + 1) * per_or
    position = {"learned": per / span, "creutz": 2 * per / span,
                "kp_overrelax": (2.5 * per + 0.5 * (N_OR + 1) * per_or) / span}
    ref_means = [b.mean() for b in blocks["kennedy_pendleton"]["P"]]
    slope, slope_err, block_err = block_drift(ref_means)
    out["equilibrium"] = {
        "reference": "Kennedy-Pendleton blocks", "blocks": nblk + 1, "sweeps_per_block": per,
        "plaquette_drift_per_round": slope, "drift_err": slope_err, "block_error": block_err,
        "drift_over_block_error": abs(slope) / block_err if block_err > 0 else None,
        "sweeps_per_round": span}
    for key, b in blocks.items():
        rate = out[key]["value"] if key != "kp_overrelax" else compound_per_s * 4 * VOL
        tp, dtp = tau_int(b["P"])[:2]
        tl, dtl = tau_int(b["L"])[:2]
        tp_own = tau_int(b["P"], own_means=True)[0]
        unit = "compound sweeps" if key == "kp_overrelax" else "sweeps"
        out[key].update({"tau_int": float(tp), "tau_int_err": float(dtp), "tau_int_abs_polyakov": float(tl),
                         "tau_int_abs_polyakov_err": float(dtl), "tau_int_own_block_means": float(tp_own),
                         "tau_int_unit": unit, "value_tau_adjusted": rate / (2 * tp),
                         "value_tau_adjusted_abs_polyakov": rate / (2 * tl),
                         "plaquette_mean": float(np.mean([x.mean() for x in b["P"]])),
                         "abs_polyakov_mean": float(np.mean([x.mean() for x in b["L"]]))})
        if key in position:
            m, se = interleaved_offset([x.mean() for x in b["P"]], ref_means, position[key])
            out[key]["plaquette_minus_kennedy_pendleton"] = m
            out[key]["plaquette_sigma"] = m / se if se > 0 else None
    out["value_tau_adjusted"] = {k: out[k]["value_tau_adjusted"] for k in blocks}
    out["value_tau_adjusted"]["convention"] = (
        "4V x sweeps/s / (2 tau_int(plaquette)), tau_int = 1/2 + sum rho in sweeps (compound sweeps for "
        "kp_overrelax), Gamma method with the interleaved blocks of a form pooled as replicas about their "
        "common mean")
    out["value_tau_adjusted_abs_polyakov"] = {k: out[k]["value_tau_adjusted_abs_polyakov"] for k in blocks}
    return out


def timed_batch(stream, torch, fn, k):
    """ms per sweep of fn(k) on the batch's stream (CUDA events), after 3 untimed sweeps."""
    fn(3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn(k)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / k


def run_batched(args, dist, su2, torch):
    """64 independent lattices (8^4, 12^3x4, 16^3x6, 16^4, 24^3x8; beta in
    [1.5, 3]; cold start): one persistent cooperative launch per sweep,
    replayed from a CUDA graph, plaquette and Polyakov loop of every lattice
    every sweep; launch shape autotuned first."""
    from paper_1010_1486_gb300 import workloads

    cfg = workloads.batched(64, seed=5 + dist.rank)
    n = len(cfg["ns"])
    sites = sum(x ** 3 * t for x, t in zip(cfg["ns"], cfg["nt"]))
    stream = torch.cuda.Stream()
    b = su2.su2_batch_create(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"], cfg["start"], stream=stream)
    try:
        su2.su2_batch_set_sampler(b, su2.SU2_SAMPLER_KP if args.sampler == "kp" else su2.SU2_SAMPLER_CREUTZ)
        su2.su2_batch_sweep(b, 20)
        # the fixed baseline first: 256-thread blocks, queue depth 4, all co-resident blocks
        su2.su2_batch_set_launch(b, 4, 256, 0)
        fixed = su2.su2_batch_launch_info(b)
        fixed_ms = timed_batch(stream, torch, lambda k: su2.su2_batch_generate(b, n, k, 1), 50)
        depth, grid = su2.su2_batch_autotune(b, 5)
        tuned = su2.su2_batch_launch_info(b)
        su2.su2_batch_generate(b, n, 5, 1)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        plaq, poly, st = su2.su2_batch_generate(b, n, args.batched_steps, 1)
        ev1.record(stream)
        ev1.synchronize()
        info = su2.su2_batch_info(b)
    finally:
        su2.su2_batch_destroy(b)
    ms = dist.reduce(ev0.elapsed_time(ev1), "max")
    updates = dist.reduce(float(st["link_updates"]), "sum")
    value = updates / (ms * 1e-3)
    peak, _ = measured_peaks()
    achieved = BYTES_PER_UPDATE * updates / dist.world / (ms * 1e-3) / 1e9
    return {"workload": "64 lattices: 8^4, 12^3x4, 16^3x6, 16^4, 24^3x8 (13/13/13/13/12), beta uniform in [1.5, 3], "
                        "cold start, plaquette and Polyakov loop of every lattice every sweep",
            "sampler": SAMPLERS[args.sampler]["name"],
            "sites": sites, "value": value, "unit": UNIT, "sweeps_per_s": args.batched_steps / (ms * 1e-3),
            "ms_per_sweep": ms / args.batched_steps,
            "autotuned": {"queue_depth": tuned[0], "threads_per_block": tuned[1], "grid_blocks": tuned[2],
                          "search": "queue depth 1/2/4/8 x 64/128/256 threads x all co-resident blocks or 1/2, "
                                    "1/4, 1/8, 1/16 of them, 5 sweeps each"},
            "fixed_config": {"queue_depth": fixed[0], "threads_per_block": fixed[1], "grid_blocks": fixed[2],
                             "ms_per_sweep": fixed_ms},
            "autotuned_speedup_vs_fixed": fixed_ms / (ms / args.batched_steps),
            "cuda_graph": info["graphs"], "gpu_launches": args.batched_steps,
            "roofline": {"bound": "hbm", "kernel": "batch_sweep_kernel", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "note": "whole sweep incl. barriers and measurements; 169 MB of links, partly L2-resident"},
            "plaquette_last": [float(x) for x in plaq[-1][:5]]}


def run_slabs(args, dist, su2, torch, lattice_sweep_s):
    """The paper's multi-GPU decomposition (Sec. 4, Fig. 1) on one GPU: the
    48^4 lattice as two time slabs of 24 slices (+ 2 ghost slices each), each
    slab on its own stream, Kennedy-Pendleton phases on the interiors and,
    after every phase, the boundary slices that phase changed copied into
    the neighbour's ghosts (device copies).  Host-timed over `slabs` sweeps
    after 3 untimed ones, against the single lattice's unmeasured sweep."""
    from paper_1010_1486_gb300.slab import LocalSlabs

    streams = [torch.cuda.Stream() for _ in range(2)]
    ls = LocalSlabs(NS, NT, 2, BETA, SEED + dist.rank, su2.SU2_HOT, streams=streams)
    try:
        ls.set_sampler(su2.SU2_SAMPLER_KP)
        ls.sweep(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ls.sweep(args.slabs)
        torch.cuda.synchronize()
        s = dist.reduce(time.perf_counter() - t0, "max") / args.slabs
        exch = su2.su2_slab_boundary_bytes(ls.h[0])
    finally:
        ls.close()
    return {"workload": "48^4, beta 6.0, hot start, two time slabs of 24 slices on one GPU (own stream each), "
                        "Kennedy-Pendleton, boundary slices copied after every phase",
            "sweeps_per_s": 1.0 / s, "ms_per_sweep": s * 1e3,
            "link_updates_per_s": dist.reduce(float(LINKS), "sum") / s,
            "vs_single_lattice_unmeasured": lattice_sweep_s / s,
            "bytes_per_boundary_slice": exch, "boundary_slices_per_phase": 4,
            "timing": "host clock around the sweeps, synchronised on both sides (the two streams)"}


def run_small(args, dist, su2, torch):
    """The small workloads, L2-resident, so latency- rather than HBM-bound:
    sweeps/s and microseconds per phase (graph-replayed sweeps on a stream,
    CUDA events around the whole run, measurements included).
      8^4, beta = 2.3, hot start (seed 1): 1000 sweeps, plaquette and
        Polyakov loop every sweep, the headline sampler;
      24^4, beta = 2.5, cold start (seed 2): 200 thermalisation sweeps, then
        1000 measured sweeps with reunitarization every 10;
      32^3 x 4, beta = 2.20 .. 2.60 in steps of 0.05, cold starts (seeds
        100 + i): one batch of nine lattices, launch shape autotuned after the
        500 thermalisation sweeps, then 2000 measured sweeps, plaquette and
        |L| per beta (Sec. 4.2)."""
    import numpy as np

    from paper_1010_1486_gb300 import workloads

    sampler = su2.SU2_SAMPLER_KP if args.sampler == "kp" else su2.SU2_SAMPLER_CREUTZ
    out = {}

    def lattice_run(cfg, therm, n, reunit):
        st_ = torch.cuda.Stream()
        h = su2.su2_create(cfg["ns"], cfg["nt"], cfg["beta"], cfg["seed"] + dist.rank, cfg["start"], stream=st_)
        try:
            su2.su2_set_sampler(h, sampler)
            su2.su2_generate(h, max(therm, 3), 1, reunit)
            ms, (plaq, poly, _) = timed(st_, torch, dist, lambda: su2.su2_generate(h, n, 1, reunit))
        finally:
            su2.su2_destroy(h)
        return ms, plaq, poly

    c1 = workloads.PARITY_8
    ms, plaq, poly = lattice_run(c1, 10, 1000, 0)
    out["8^4"] = {"workload": "8^4, beta 2.3, hot start, 1000 sweeps, plaquette + Polyakov loop every sweep",
                  "sweeps_per_s": 1000 / (ms * 1e-3), "us_per_phase": ms * 1e3 / (8 * 1000),
                  "link_updates_per_s": 1000 * 4 * 8 ** 4 / (ms * 1e-3), "plaquette_mean": float(plaq.mean())}
    c2 = workloads.SCALE_24
    ms, plaq, poly = lattice_run(c2, c2["therm"], c2["meas"], c2["reunit_every"])
    out["24^4"] = {"workload": "24^4, beta 2.5, cold start, 200 + 1000 sweeps, reunitarized every 10, plaquette "
                               "(binary64 sum) every sweep",
                   "sweeps_per_s": c2["meas"] / (ms * 1e-3), "us_per_phase": ms * 1e3 / (8 * c2["meas"]),
                   "link_updates_per_s": c2["meas"] * 4 * 24 ** 4 / (ms * 1e-3),
                   "plaquette_mean": float(plaq.mean())}
    c4 = workloads.FINITE_T
    nb = len(c4["betas"])
    bst = torch.cuda.Stream()
    b = su2.su2_batch_create([c4["ns"]] * nb, [c4["nt"]] * nb, list(c4["betas"]),
                             [c4["seed0"] + i for i in range(nb)], c4["start"], stream=bst)
    try:
        su2.su2_batch_set_sampler(b, sampler)
        su2.su2_batch_generate(b, nb, 500, 0)
        su2.su2_batch_autotune(b, 5)  # restores the links and the sweep counter
        scan_launch = su2.su2_batch_launch_info(b)
        ms, (plaq, poly, _) = timed(bst, torch, dist, lambda: su2.su2_batch_generate(b, nb, 2000, 1))
    finally:
        su2.su2_batch_destroy(b)
    out["32^3x4_beta_scan"] = {
        "workload": "nine 32^3 x 4 lattices, beta 2.20 .. 2.60, cold, one batch (headline sampler): 500 + 2000 "
                    "sweeps, plaquette and Polyakov loop of every lattice every sweep",
        "sweeps_per_s": 2000 / (ms * 1e-3), "us_per_sweep_of_the_scan": ms * 1e3 / 2000,
        "link_updates_per_s": 2000 * nb * 4 * 32 ** 3 * 4 / (ms * 1e-3),
        "autotuned": {"queue_depth": scan_launch[0], "threads_per_block": scan_launch[1],
                      "grid_blocks": scan_launch[2]},
        "beta": list(c4["betas"]), "plaquette_mean": [float(x) for x in plaq.mean(axis=0)],
        "abs_polyakov_mean": [float(x) for x in np.abs(poly).mean(axis=0)]}
    out["32^3x4_beta_scan_learned"] = run_scan_learned(args, dist, su2, torch, c4,
                                                       out["32^3x4_beta_scan"]["plaquette_mean"])
    return out


def run_scan_learned(args, dist, su2, torch, c4, plain_plaquette):
    """The beta scan with the learned proposal and its plain fallback: the
    nine 32^3 x 4 lattices (cold, seeds 100 + i) thermalised by 500
    Kennedy-Pendleton sweeps each, one network trained on (beta k, a0) pairs
    pooled over the scan (10^5 per lattice, 1500 + 1500 Adam steps), then
    2000 measured sweeps per lattice with the proposal (fallback below 0.7
    acceptance), the lattices one after another on one stream."""
    import numpy as np

    from paper_1010_1486_gb300 import learn

    nb = len(c4["betas"])
    ns, nt = c4["ns"], c4["nt"]
    st_ = torch.cuda.Stream()
    lats = [su2.su2_create(ns, nt, b, c4["seed0"] + i + dist.rank, c4["start"], stream=st_)
            for i, b in enumerate(c4["betas"])]
    try:
        for h in lats:
            su2.su2_set_sampler(h, su2.SU2_SAMPLER_KP)
            su2.su2_generate(h, 500, 0, 0)
        pairs = torch.cat([learn.collect(h, ns, nt, 100_000) for h in lats])
        w, _, s_lo, s_hi = learn.train(pairs, steps=1500, batch=8192, lr=3e-3, seed=4, tail_steps=1500, tail_lr=3e-4)
        del pairs
        for h in lats:
            su2.su2_set_proposal(h, w, s_lo, s_hi, 256)
            su2.su2_learned_generate(h, 3, 1, 0.7)
        res = []
        ms, _ = timed(st_, torch, dist, lambda: [res.append(su2.su2_learned_generate(h, 2000, 1, 0.7)) for h in lats])
    finally:
        for h in lats:
            su2.su2_destroy(h)
    acc = [sum(r[2]["accepted"]) / max(1, r[2]["learned_sweeps"] * 4 * ns ** 3 * nt) for r in res]
    return {"workload": "nine 32^3 x 4 lattices, beta 2.20 .. 2.60, cold, 500 Kennedy-Pendleton sweeps each, one "
                        "network trained on pairs pooled over the scan, then 2000 learned sweeps (fallback below "
                        "0.7 acceptance) per lattice, one after another, plaquette and Polyakov loop every sweep",
            "sweeps_per_s": 2000 * nb / (ms * 1e-3), "us_per_sweep": ms * 1e3 / (2000 * nb),
            "sweeps_of_the_scan_per_s": 2000 / (ms * 1e-3),
            "acceptance": [float(a) for a in acc],
            "learned_sweeps": [int(r[2]["learned_sweeps"]) for r in res],
            "fallback_sweeps": [int(r[2]["plain_sweeps"]) for r in res],
            "plaquette_mean": [float(np.mean(r[0])) for r in res],
            "plaquette_minus_plain_batch": [float(np.mean(r[0])) - float(p) for r, p in zip(res, plain_plaquette)],
            "abs_polyakov_mean": [float(np.mean(np.abs(r[1]))) for r in res]}


def run_e2e(args, dist, lat, su2, torch):
    """Per step: a configuration in from pinned host memory, one sweep with
    plaquette and Polyakov loop read back, the new configuration out to
    pinned host memory -- through the C ABI's asynchronous calls
    (su2_set_links_async, su2_generate_async, su2_get_links_async, su2_sync).
    --e2e-in-flight configurations (default 4) are in flight, each on its own
    lattice handle and stream, taken round robin: the copy engines move one configuration while
    another is swept.  Each handle's output is its next input, so every
    handle runs its own chain (seeds differ) through host memory.  All copies
    of all steps are inside the timed region.  Three timed repetitions of
    e2e_steps steps each; the value is their median (the host link of the
    virtual machines this runs on varies from run to run), all three are
    reported."""
    start = su2.su2_get_links(lat, NS, NT)
    hs, bufs, meas = [], [], []
    try:
        for i in range(args.e2e_in_flight):
            hs.append(su2.su2_create(NS, NT, BETA, SEED + dist.rank + 1000 * (i + 1), su2.SU2_COLD,
                                     stream=torch.cuda.Stream()))
            a = torch.empty((VOL, 4, 4), dtype=torch.float32, pin_memory=True).numpy()
            b = torch.empty((VOL, 4, 4), dtype=torch.float32, pin_memory=True).numpy()
            a[...] = start
            bufs.append([a, b])
            meas.append(torch.empty(2, dtype=torch.float64, pin_memory=True).numpy())

        def step(i):
            h = hs[i]
            su2.su2_sync(h)  # its previous step is done: that output is this input
            bufs[i].reverse()
            su2.su2_set_links_async(h, bufs[i][0])
            su2.su2_generate_async(h, 1, 1, 0, meas[i][0:1], meas[i][1:2])
            su2.su2_get_links_async(h, bufs[i][1])

        for i in range(args.e2e_in_flight):  # untimed: staging buffers, graph capture
            bufs[i].reverse()
            step(i)
        for h in hs:
            su2.su2_sync(h)
        reps = []
        for _ in range(3):
            dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(args.e2e_steps):
                step(k % args.e2e_in_flight)
            for h in hs:
                su2.su2_sync(h)
            reps.append(dist.reduce(time.perf_counter() - t0, "max"))
        e2e_s = statistics.median(reps)
    finally:
        for h in hs:
            su2.su2_destroy(h)
    e2e_updates = dist.reduce(float(args.e2e_steps * LINKS), "sum")
    return {"value": e2e_updates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": LINKS * 16,
            "d2h_bytes_per_step": LINKS * 16 + 16, "steps": args.e2e_steps,
            "ms_per_step": e2e_s * 1e3 / args.e2e_steps,
            "repetitions": [e2e_updates / r for r in reps], "statistic": "median of 3 timed repetitions",
            "pipeline": f"{args.e2e_in_flight} configurations in flight (own lattice handle and stream each, round "
                        "robin); host<->device copies on the copy engines overlap the other configurations' "
                        "sweeps"}


# --------------------------------------------------------- oracle timings
def oracle_sample(seconds: float, label: str):
    """The CPU oracle, as it stands, on the same lattice: untimed hot start,
    then whole steps (sweep over all host cores + plaquette + Polyakov loop)
    until `seconds` have passed."""
    import oracle

    threads = oracle.max_threads()
    links = oracle.hot_start(NS, NT, SEED)
    steps = 0
    t0 = time.perf_counter()
    while True:
        oracle.heatbath_sweep(NS, NT, BETA, SEED, steps, links, nthreads=threads)
        oracle.plaquette(NS, NT, links)
        oracle.polyakov(NS, NT, links)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    # one core, the paper's serial-CPU comparison: one even/odd phase (V/2 updates)
    t1 = time.perf_counter()
    oracle.heatbath_phase(NS, NT, BETA, SEED, steps, 0, 0, links, nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": steps * LINKS / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{label}: {steps} step(s) of the {NS}^4 beta={BETA} hot-start lattice "
                      f"(one sweep over {threads} threads + plaquette + Polyakov loop), {dt:.1f} s",
            "single_core": {"value": (LINKS // 8) / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"one even/odd phase ({LINKS // 8} link updates) of the same lattice on "
                                      f"one thread, {dt1:.1f} s"}}


def run_reference(args, world: int):
    """Reference arm: the CPU oracle on the same workload.  A step is one
    even/odd phase (V/2 link updates, the 8 phases cycling as in a sweep);
    after every 8th step (a full sweep) the plaquette and Polyakov loop are
    computed, so K steps stay within a few minutes."""
    import oracle

    threads = oracle.max_threads()
    links = oracle.hot_start(NS, NT, SEED)
    phases = [(mu, p) for mu in range(4) for p in range(2)]

    def step(k):
        mu, p = phases[k % 8]
        oracle.heatbath_phase(NS, NT, BETA, SEED, k // 8, mu, p, links, nthreads=threads)
        if k % 8 == 7:
            oracle.plaquette(NS, NT, links)
            oracle.polyakov(NS, NT, links)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        step(k)
    dt = time.perf_counter() - t0
    value = args.steps * (VOL // 2) / dt
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_RATE, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{NS}^4 lattice, beta={BETA}, hot start (Philox seed {SEED}); reference step = one "
                               "even/odd heat-bath phase, plaquette + Polyakov loop after every 8th step",
                   "lattice": [NS, NS, NS, NT], "beta": BETA, "start": "hot", "form": "CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} phases ({args.steps * (VOL // 2)} link updates) after "
                                   f"{args.warmup} warm-up phases"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        # rank 0 alone times the oracle; other ranks exit without work
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(run_reference(args, int(os.environ.get("WORLD_SIZE", "1")))), flush=True)
        return 0
    dist = Dist(args.gpus)
    try:
        result = run_ours(args, dist)
        if dist.rank == 0:
            if dist.world == 1 and not args.no_cpu_baseline:
                result["cpu_baseline"] = oracle_sample(args.cpu_seconds, "bounded sample")
            else:
                result["cpu_baseline"] = None
            print(json.dumps(result), flush=True)
        return 0
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
