"""Writes oracle_chains.txt: short chains of the CPU oracle recorded digit
for digit, so any change to the oracle's arithmetic shows up as a diff.

The paper prints no numerical worked example (its results are figures), so
this folder holds no paper values.  The file below is not an expected value
for the CUDA path either: the GPU tests compare against the oracle run live.
It pins the oracle to itself over time, and is regenerated only when the
oracle's arithmetic changes on purpose (the commit names the reason).

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_chains.txt")


def records():
    rows = []
    # Creutz heat bath, 4^4, beta = 2.3, hot start from seed 1
    ns, nt, beta, seed = 4, 4, 2.3, 1
    links = oracle.hot_start(ns, nt, seed)
    for s in range(5):
        tr = oracle.heatbath_sweep(ns, nt, beta, seed, s, links)
        rows.append(("creutz_4x4x4x4_b2.3", s, oracle.plaquette(ns, nt, links), oracle.polyakov(ns, nt, links),
                     " ".join(str(int(t)) for t in tr)))
    # over-relaxation after it
    for s in range(2):
        oracle.overrelax_sweep(ns, nt, links)
        rows.append(("overrelax_4x4x4x4", s, oracle.plaquette(ns, nt, links), oracle.polyakov(ns, nt, links), "-"))
    w = oracle.wilson_loops(ns, nt, links, 2, 2)
    rows.append(("wilson_2x2", 0, float(w[0, 0]), float(w[1, 1]), f"{float(w[0, 1])!r} {float(w[1, 0])!r}"))
    # Kennedy-Pendleton, 4^3 x 6, beta = 6.0, hot start from seed 2
    ns, nt, beta, seed = 4, 6, 6.0, 2
    links = oracle.hot_start(ns, nt, seed)
    for s in range(3):
        tr = oracle.heatbath_sweep_kp(ns, nt, beta, seed, s, links)
        rows.append(("kp_4x4x4x6_b6", s, oracle.plaquette(ns, nt, links), oracle.polyakov(ns, nt, links),
                     " ".join(str(int(t)) for t in tr)))
    return rows


def render(rows):
    lines = ["# name sweep plaquette polyakov extra  (written by make_golden.py from oracle/ only)"]
    for name, s, p, l, extra in rows:
        lines.append(f"{name} {s} {float(p)!r} {float(l)!r} {extra}")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write(render(records()))
    print(OUT)
