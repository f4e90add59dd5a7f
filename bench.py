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
CUDA-event duration (events recorded by the library on the launching stream).
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
HB_SOURCES = ["paper_1010_1486_gb300/csrc/heatbath.cu", "paper_1010_1486_gb300/csrc/su2_device.cuh"]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "hb_phase_48x48x48x48_beta6.md")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--tau-sweeps", type=int, default=2000, help="extra sweeps for tau_int (0 = skip)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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


def ncu_traffic_per_launch():
    """DRAM bytes per phase launch from the committed ncu summary, if it was
    taken on the current source of the heat-bath kernel; else None."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    text = open(PROFILE_SUMMARY).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != source_digest(HB_SOURCES):
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
    lat = su2.su2_create(NS, NT, BETA, seed, su2.SU2_HOT, stream=stream)
    try:
        su2.su2_generate(lat, args.warmup, 1, 0)
        su2.su2_set_timing(lat, True)
        gpu_index = dist.local_rank
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            try:
                gpu_index = int(vis.split(",")[dist.local_rank])
            except ValueError:
                pass
        clocks = ClockSampler(gpu_index, os.path.join(tempfile.gettempdir(), f"su2_clocks_rank{dist.rank}.csv"))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        ev0.record(stream)
        plaq, poly, st = su2.su2_generate(lat, args.steps, 1, 0)
        ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        clk = clocks.stop()
        dist.barrier()
        ms = ev0.elapsed_time(ev1)
        su2.su2_set_timing(lat, False)
        ms_max = dist.reduce(ms, "max")
        updates = dist.reduce(float(st["link_updates"]), "sum")
        value = updates / (ms_max * 1e-3)
        phase_s = st["kernel_ms"] / st["kernel_launches"] * 1e-3
        peak, peak_kind = measured_peaks()
        achieved = BYTES_PER_UPDATE * (VOL // 2) / phase_s / 1e9
        trials_per_update = sum(st["trials"]) / st["link_updates"]

        # end to end through the C ABI with host buffers
        e2e = None
        if args.e2e_steps > 0:
            e2e = run_e2e(args, dist, lat, su2, torch)

        tau = None
        if args.tau_sweeps > 0:
            tp, _, _ = su2.su2_generate(lat, args.tau_sweeps, 1, 0)
            half = tp[len(tp) // 2:]
            t, dt, w, err = tau_int(half)
            tau = {"observable": "plaquette", "sweeps": len(half), "tau_int": t, "tau_int_err": dt,
                   "plaquette_mean": float(np.mean(half)), "plaquette_err": err,
                   "value_tau_adjusted": value / (2.0 * t)}
    finally:
        su2.su2_destroy(lat)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_RATE, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{NS}^4 lattice, beta={BETA}, hot start (Philox seed {SEED}+rank), one step = "
                               "heat-bath sweep (8 even/odd phases) + plaquette + Polyakov loop",
                   "lattice": [NS, NS, NS, NT], "beta": BETA, "start": "hot", "form": "plain heat bath (Creutz)",
                   "parallelism": "independent replicas" if dist.world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (340 MB of links vs 129 MB L2), no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic_per_launch(), "kernel": "hb_phase_kernel",
                     "peak_source": f"{peak_kind} hbm_gbs", "bytes_per_launch": BYTES_PER_UPDATE * (VOL // 2),
                     "avg_launch_us": phase_s * 1e6},
        "e2e": e2e,
        "gpu_launches": st["kernel_launches"] + 2 * args.steps,
        "clocks": clk,
        "trials_per_update": trials_per_update,
        "plaquette_last": float(plaq[-1]), "polyakov_last": float(poly[-1]),
        "tau_int": tau,
    }
    return result


def run_e2e(args, dist, lat, su2, torch):
    """Per step: configuration in from pinned host memory (su2_set_links), one
    sweep with plaquette and Polyakov loop read back (su2_generate), the new
    configuration out to pinned host memory (su2_get_links)."""
    pin_a = torch.empty((VOL, 4, 4), dtype=torch.float32, pin_memory=True).numpy()
    pin_b = torch.empty((VOL, 4, 4), dtype=torch.float32, pin_memory=True).numpy()
    su2.su2_get_links(lat, NS, NT, out=pin_a)
    p_host = torch.empty(1, dtype=torch.float64, pin_memory=True).numpy()
    l_host = torch.empty(1, dtype=torch.float64, pin_memory=True).numpy()
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        su2.su2_set_links(lat, pin_a)
        su2.su2_generate(lat, 1, 1, 0, plaq=p_host, poly=l_host)
        su2.su2_get_links(lat, NS, NT, out=pin_b)
        pin_a, pin_b = pin_b, pin_a
    e2e_s = dist.reduce(time.perf_counter() - t0, "max")
    e2e_updates = dist.reduce(float(args.e2e_steps * LINKS), "sum")
    return {"value": e2e_updates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": LINKS * 16,
            "d2h_bytes_per_step": LINKS * 16 + 16, "steps": args.e2e_steps,
            "ms_per_step": e2e_s * 1e3 / args.e2e_steps}


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
    return {"value": steps * LINKS / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{label}: {steps} step(s) of the {NS}^4 beta={BETA} hot-start lattice "
                      f"(one sweep over {threads} threads + plaquette + Polyakov loop), {dt:.1f} s"}


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
