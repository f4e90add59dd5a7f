"""su2_generate on a user stream replays each sweep from a captured CUDA
graph (the sweep counter and the measurement slot live in device memory);
on the legacy default stream it launches eagerly.  Both must give the same
chain bit for bit: links, plaquette and Polyakov histories, trial counts --
through every measurement / reunitarization variant and after every setting
the captured sweep depends on changes."""
import numpy as np
import pytest

from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu


def run(stream, ns, nt, script):
    h = su2.su2_create(ns, nt, 2.3, 11, su2.SU2_HOT, stream=stream)
    out = []
    try:
        for step in script:
            kind = step[0]
            if kind == "gen":
                _, n, me, re_ = step
                p, l, st = su2.su2_generate(h, n, me, re_)
                out.append((p.copy(), l.copy(), st["trials"], st["link_updates"]))
            elif kind == "sampler":
                su2.su2_set_sampler(h, step[1])
            elif kind == "or":
                su2.su2_set_overrelax(h, step[1])
            elif kind == "beta":
                su2.su2_set_beta(h, step[1])
            elif kind == "state":
                st = su2.su2_get_state(h)
                st["sweep"] += step[1]
                su2.su2_set_state(h, st)
        out.append(su2.su2_get_links(h, ns, nt))
        out.append(su2.su2_get_state(h)["sweep"])
    finally:
        su2.su2_destroy(h)
    return out


SCRIPT = [("gen", 7, 1, 0), ("gen", 9, 2, 3), ("gen", 6, 3, 2), ("sampler", su2.SU2_SAMPLER_KP), ("gen", 5, 1, 0),
          ("or", 2), ("gen", 4, 1, 4), ("beta", 2.6), ("gen", 5, 1, 0), ("or", 0), ("sampler", su2.SU2_SAMPLER_CREUTZ),
          ("state", 100), ("gen", 3, 1, 1), ("gen", 1, 1, 0), ("gen", 4, 0, 0), ("gen", 12, 1, 0)]  # last: history grows


@pytest.mark.parametrize("ns,nt", [(8, 8), (6, 4), (2, 2)])
def test_graph_replays_equal_eager_launches(ns, nt):
    import torch

    eager = run(None, ns, nt, SCRIPT)
    graphs = run(torch.cuda.Stream(), ns, nt, SCRIPT)
    for a, b in zip(eager[:-2], graphs[:-2]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert a[2] == b[2] and a[3] == b[3]
    assert np.array_equal(eager[-2], graphs[-2])
    assert eager[-1] == graphs[-1]


def test_timing_keeps_eager_launches_on_a_user_stream():
    import torch

    h = su2.su2_create(8, 4, 2.3, 3, su2.SU2_HOT, stream=torch.cuda.Stream())
    try:
        su2.su2_set_timing(h, True)
        st = su2.su2_heatbath_sweep(h, 3, stats=True)
        assert st["timed"] and st["kernel_ms"] > 0
    finally:
        su2.su2_destroy(h)
