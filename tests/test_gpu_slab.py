"""Time slabs on the GPU (Sec. 4, multi-GPU part; Fig. 1), through the C ABI.

A lattice split into time slabs, each with two ghost slices, that exchange the
boundary links after every phase must reproduce the single lattice's chain bit
for bit (the random numbers are keyed by the global site), with the same trial
counts.  Checked for slabs in one process (device-to-device exchange), for
boundaries moved through host buffers, and for two processes on one GPU that
exchange through torch.distributed (gloo), as ranks on separate GPUs would.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import slab as slabmod
from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu


def slab_from(full, ext):
    sl = full.reshape(ext.nt, ext.ns ** 3, 4, 4)
    idx = [(ext.t0 - 1 + tl) % ext.nt for tl in range(ext.nt_local + 2)]
    return np.ascontiguousarray(sl[idx].reshape(-1, 4, 4))


def interior(local, ext):
    vs = ext.ns ** 3
    return local[vs:(ext.nt_local + 1) * vs]


def lattice_chain(ns, nt, beta, seed, sweeps, sampler):
    h = su2.su2_create(ns, nt, beta, seed, su2.SU2_HOT)
    try:
        su2.su2_set_sampler(h, sampler)
        st = su2.su2_heatbath_sweep(h, sweeps, stats=True)
        return su2.su2_get_links(h, ns, nt), st["trials"]
    finally:
        su2.su2_destroy(h)


def test_slab_hot_start_is_the_lattice_hot_start():
    ns, nt, seed = 4, 8, 3
    full = oracle.hot_start(ns, nt, seed)
    for r in range(2):
        ext = slabmod.slab_extent(ns, nt, r, 2)
        h = su2.su2_slab_create(ns, nt, ext.t0, ext.nt_local, 2.0, seed, su2.SU2_HOT)
        try:
            assert np.array_equal(su2.su2_slab_get_links(h, ns, ext.nt_local), slab_from(full, ext))
            assert su2.su2_slab_info(h) == (ext.t0, ext.nt_local, 0)
        finally:
            su2.su2_slab_destroy(h)


@pytest.mark.parametrize("ns,nt,nslabs,sampler,beta", [
    (8, 8, 2, su2.SU2_SAMPLER_CREUTZ, 2.3),
    (8, 8, 1, su2.SU2_SAMPLER_KP, 6.0),
    (6, 12, 3, su2.SU2_SAMPLER_KP, 2.5),
    (16, 16, 4, su2.SU2_SAMPLER_CREUTZ, 6.0),
    (48, 48, 2, su2.SU2_SAMPLER_KP, 6.0),
])
def test_slabs_in_one_process_equal_the_lattice(ns, nt, nslabs, sampler, beta):
    seed, sweeps = 11, 2
    want, want_trials = lattice_chain(ns, nt, beta, seed, sweeps, sampler)
    slabs = slabmod.LocalSlabs(ns, nt, nslabs, beta, seed, su2.SU2_HOT)
    try:
        slabs.set_sampler(sampler)
        slabs.sweep(sweeps)
        parts, trials = [], np.zeros(8, dtype=np.int64)
        for h, ext in zip(slabs.h, slabs.extents):
            local = su2.su2_slab_get_links(h, ns, ext.nt_local)
            assert np.array_equal(local, slab_from(want, ext))  # ghosts current too
            parts.append(interior(local, ext))
            t, fails = su2.su2_slab_stats(h)
            trials += np.array(t)
            assert fails == 0
    finally:
        slabs.close()
    assert np.array_equal(np.concatenate(parts), want)
    assert [int(t) for t in trials] == [int(t) for t in want_trials]


def test_slabs_on_their_own_streams_equal_the_lattice():
    torch = pytest.importorskip("torch")
    ns, nt, beta, seed = 8, 12, 2.4, 5
    want, _ = lattice_chain(ns, nt, beta, seed, 2, su2.SU2_SAMPLER_CREUTZ)
    streams = [torch.cuda.Stream() for _ in range(3)]
    slabs = slabmod.LocalSlabs(ns, nt, 3, beta, seed, su2.SU2_HOT, streams=streams)
    try:
        slabs.sweep(2)
        got = np.concatenate([interior(su2.su2_slab_get_links(h, ns, e.nt_local), e)
                              for h, e in zip(slabs.h, slabs.extents)])
    finally:
        slabs.close()
    assert np.array_equal(got, want)


def test_boundaries_through_host_buffers_equal_the_lattice():
    """The multi-process path in one process: pack to host, unpack from host."""
    ns, nt, beta, seed, nslabs = 8, 8, 2.3, 9, 2
    want, _ = lattice_chain(ns, nt, beta, seed, 1, su2.SU2_SAMPLER_CREUTZ)
    exts = [slabmod.slab_extent(ns, nt, r, nslabs) for r in range(nslabs)]
    hs = [su2.su2_slab_create(ns, nt, e.t0, e.nt_local, beta, seed, su2.SU2_HOT) for e in exts]
    try:
        nbytes = su2.su2_slab_boundary_bytes(hs[0])
        assert nbytes == 8 * ns ** 3
        bufs = [[np.zeros(nbytes // 4, np.float32) for _ in range(2)] for _ in hs]
        for mu, parity in slabmod.PHASES:
            for h in hs:
                su2.su2_slab_phase(h, mu, parity)
            for h, b in zip(hs, bufs):
                su2.su2_slab_pack(h, mu, parity, slabmod.FIRST, b[0].ctypes.data)
                su2.su2_slab_pack(h, mu, parity, slabmod.LAST, b[1].ctypes.data)
                su2.su2_slab_sync(h)
            for r, h in enumerate(hs):
                lo, hi = slabmod.neighbours(r, nslabs)
                su2.su2_slab_unpack(h, mu, parity, slabmod.LOWER_GHOST, bufs[lo][1].ctypes.data)
                su2.su2_slab_unpack(h, mu, parity, slabmod.UPPER_GHOST, bufs[hi][0].ctypes.data)
                su2.su2_slab_sync(h)
        got = np.concatenate([interior(su2.su2_slab_get_links(h, ns, e.nt_local), e) for h, e in zip(hs, exts)])
    finally:
        for h in hs:
            su2.su2_slab_destroy(h)
    assert np.array_equal(got, want)


def test_slab_arguments_are_checked():
    for args in [(8, 8, 1, 4), (8, 8, 0, 3), (8, 8, 6, 4), (7, 8, 0, 4), (8, 8, -2, 4)]:
        with pytest.raises(su2.SU2Error):
            su2.su2_slab_create(*args, 2.0, 1, su2.SU2_COLD)
    a = su2.su2_slab_create(4, 8, 0, 2, 2.0, 1, su2.SU2_COLD)
    b = su2.su2_slab_create(4, 8, 4, 2, 2.0, 1, su2.SU2_COLD)
    try:
        with pytest.raises(su2.SU2Error):
            su2.su2_slab_exchange(a, b, 0, 0)  # not neighbours: slices 0-1 and 4-5
        with pytest.raises(su2.SU2Error):
            su2.su2_slab_phase(a, 4, 0)
    finally:
        su2.su2_slab_destroy(a)
        su2.su2_slab_destroy(b)


# ------------------------------------------------- two processes, one GPU
NS, NT, BETA, SEED, SWEEPS = 8, 8, 2.3, 13, 2


def _rank_main(rank, world, port, outdir):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = slabmod.DistributedSlab(NS, NT, BETA, SEED, su2.SU2_HOT)
        try:
            s.sweep(SWEEPS)
            local = su2.su2_slab_get_links(s.h, NS, s.extent.nt_local)
            np.save(os.path.join(outdir, f"interior{rank}.npy"), interior(local, s.extent))
        finally:
            s.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_two_processes_exchanging_through_gloo_equal_the_lattice():
    mp = pytest.importorskip("torch.multiprocessing")
    want, _ = lattice_chain(NS, NT, BETA, SEED, SWEEPS, su2.SU2_SAMPLER_CREUTZ)
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True)
        got = np.concatenate([np.load(os.path.join(d, f"interior{r}.npy")) for r in range(2)])
    assert np.array_equal(got, want)
