"""Host logic of bench.py: rank aggregation over a world-size-2 gloo group on
the CPU, and the reference arm's JSON line (the CPU oracle)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
d = bench.Dist(2)
mx = d.reduce(float(d.rank + 1) * 10.0, "max")
sm = d.reduce(float(d.rank + 1), "sum")
d.barrier()
print(json.dumps({{"rank": d.rank, "max": mx, "sum": sm}}))
d.close()
"""


def test_two_rank_gloo_reduction():
    pytest.importorskip("torch")
    port = _free_port()
    code = WORKER.format(root=ROOT)
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda r: r["rank"])
    assert [r["max"] for r in res] == [20.0, 20.0]
    assert [r["sum"] for r in res] == [3.0, 3.0]


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "cpu_baseline", "e2e", "config"):
        assert key in line, key
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], capture_output=True,
                       text=True, timeout=120, env=env, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_nvml_clock_sampler_summary_with_a_fake_library():
    """The in-window clock record: median SM clock, the maximum, and the
    clock-event reasons decoded from NVML's bit mask, from a fake NVML."""
    import threading

    sys.path.insert(0, ROOT)
    import bench

    class Fake:
        def __init__(self):
            self.n = 0

        def nvmlDeviceGetClockInfo(self, h, kind, ref):
            self.n += 1
            ref._obj.value = 2070 if self.n % 3 else 1980
            return 0

        def nvmlDeviceGetMaxClockInfo(self, h, kind, ref):
            ref._obj.value = 2070
            return 0

        def nvmlDeviceGetPowerUsage(self, h, ref):
            ref._obj.value = 950000
            return 0

        def nvmlShutdown(self):
            return 0

    fake = Fake()
    s = object.__new__(bench.NvmlClockSampler)
    import ctypes

    s.ct, s.lib, s.h = ctypes, fake, None
    s.reasons_fn = lambda h, ref: setattr(ref._obj, "value", 0x4 | 0x1) or 0
    s.rows, s.done = [], threading.Event()
    for _ in range(6):
        s._sample()
    s.thread = threading.Thread(target=lambda: None)
    s.thread.start()
    out = s.stop()
    assert out["samples"] == 6 and out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2070.0 and out["reasons"] == ["sw_power_cap"]
    assert abs(out["power_w_max"] - 950.0) < 1e-9
