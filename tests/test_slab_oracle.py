"""Time-slab decomposition (Sec. 4, multi-GPU part; Fig. 1) on the CPU.

The oracle runs each rank's phases on its slab (interior slices plus two
ghost slices); after every phase the boundary slices' changed links move to
the neighbours' ghosts following the package's exchange plan.  The random
numbers are keyed by the global site, so the decomposed chain must equal the
single-lattice oracle chain bit for bit, trial counts included.  One test
runs the slabs in one process; another runs two gloo ranks that exchange
through torch.distributed point-to-point messages.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
from paper_1010_1486_gb300 import slab as slabmod


def slab_from(full, ext):
    """The slab's local array from the full lattice: local slice tl is global
    slice (t0 - 1 + tl) mod nt."""
    vs = ext.ns ** 3
    sl = full.reshape(ext.nt, vs, 4, 4)
    idx = [(ext.t0 - 1 + tl) % ext.nt for tl in range(ext.nt_local + 2)]
    return np.ascontiguousarray(sl[idx].reshape(-1, 4, 4))


def parity_sites(ext, tl, parity):
    """Sites of local slice tl whose global parity is `parity`."""
    ns = ext.ns
    tg = (ext.t0 - 1 + tl) % ext.nt
    x, y, z = np.meshgrid(np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij")
    lex = ((z * ns + y) * ns + x).ravel()
    keep = ((x + y + z).ravel() + tg) % 2 == parity
    return tl * ns ** 3 + np.sort(lex[keep])


def pack(slab, ext, mu, parity, side):
    tl = 1 if side == slabmod.FIRST else ext.nt_local
    return slab[parity_sites(ext, tl, parity), mu, :].copy()


def unpack(slab, ext, mu, parity, side, buf):
    tl = 0 if side == slabmod.LOWER_GHOST else ext.nt_local + 1
    slab[parity_sites(ext, tl, parity), mu, :] = buf


def interior(slab, ext):
    vs = ext.ns ** 3
    return slab[vs:(ext.nt_local + 1) * vs]


def full_chain(ns, nt, beta, seed, sweeps, kp):
    links = oracle.hot_start(ns, nt, seed)
    trials = np.zeros(8, dtype=np.int64)
    for s in range(sweeps):
        f = oracle.heatbath_sweep_kp if kp else oracle.heatbath_sweep
        trials += f(ns, nt, beta, seed, s, links)
    return links, trials


def test_exchange_plan_pairs_every_send_with_a_receive():
    for world in (1, 2, 3, 4, 6):
        sends, recvs = [], []
        for r in range(world):
            for kind, peer, side, tag in slabmod.exchange_plan(r, world):
                (sends if kind == "send" else recvs).append((r, peer, side, tag))
        assert len(sends) == len(recvs) == 2 * world
        for r, peer, side, tag in sends:
            # the receiver expects this tag from r, into the ghost the side feeds
            ghost = slabmod.UPPER_GHOST if side == slabmod.FIRST else slabmod.LOWER_GHOST
            assert (peer, r, ghost, tag) in recvs
        lo, hi = slabmod.neighbours(0, world)
        assert lo == world - 1 and hi == 1 % world


def test_slab_extents():
    e = slabmod.slab_extent(4, 12, 2, 3)
    assert (e.t0, e.nt_local) == (8, 4)
    with pytest.raises(ValueError):
        slabmod.slab_extent(4, 12, 0, 4)  # 3 slices: odd
    with pytest.raises(ValueError):
        slabmod.slab_extent(4, 12, 0, 5)


@pytest.mark.parametrize("ns,nt,nslabs,kp", [(4, 8, 2, False), (4, 12, 3, True), (6, 4, 2, False),
                                             (4, 8, 1, True), (4, 8, 4, False)])
def test_slabs_in_one_process_equal_the_lattice_chain(ns, nt, nslabs, kp):
    beta, seed, sweeps = (6.0 if kp else 2.3), 5, 2
    want, want_trials = full_chain(ns, nt, beta, seed, sweeps, kp)
    start = oracle.hot_start(ns, nt, seed)
    exts = [slabmod.slab_extent(ns, nt, r, nslabs) for r in range(nslabs)]
    slabs = [slab_from(start, e) for e in exts]
    trials = np.zeros(8, dtype=np.int64)
    for s in range(sweeps):
        for mu, parity in slabmod.PHASES:
            for e, sl in zip(exts, slabs):
                trials[2 * mu + parity] += oracle.slab_phase(ns, nt, e.t0, e.nt_local, beta, seed, s, mu, parity,
                                                             sl, kp=kp)
            out = [{side: pack(sl, e, mu, parity, side) for side in (slabmod.FIRST, slabmod.LAST)}
                   for e, sl in zip(exts, slabs)]
            for r, (e, sl) in enumerate(zip(exts, slabs)):
                lo, hi = slabmod.neighbours(r, nslabs)
                unpack(sl, e, mu, parity, slabmod.LOWER_GHOST, out[lo][slabmod.LAST])
                unpack(sl, e, mu, parity, slabmod.UPPER_GHOST, out[hi][slabmod.FIRST])
    got = np.concatenate([interior(sl, e) for e, sl in zip(exts, slabs)])
    assert np.array_equal(got, want)
    assert np.array_equal(trials, want_trials)
    # the ghosts hold the neighbours' current boundary slices
    for e, sl in zip(exts, slabs):
        assert np.array_equal(sl, slab_from(want, e))


def test_a_slab_phase_without_the_exchange_differs():
    """Planted mistake: skipping the exchange after one phase changes the
    chain (the ghosts are read by the next phase)."""
    ns, nt, beta, seed = 4, 8, 2.3, 5
    want, _ = full_chain(ns, nt, beta, seed, 1, False)
    start = oracle.hot_start(ns, nt, seed)
    exts = [slabmod.slab_extent(ns, nt, r, 2) for r in range(2)]
    slabs = [slab_from(start, e) for e in exts]
    for mu, parity in slabmod.PHASES:
        for e, sl in zip(exts, slabs):
            oracle.slab_phase(ns, nt, e.t0, e.nt_local, beta, seed, 0, mu, parity, sl)
        if (mu, parity) == (1, 0):
            continue
        out = [{side: pack(sl, e, mu, parity, side) for side in (slabmod.FIRST, slabmod.LAST)}
               for e, sl in zip(exts, slabs)]
        for r, (e, sl) in enumerate(zip(exts, slabs)):
            lo, hi = slabmod.neighbours(r, 2)
            unpack(sl, e, mu, parity, slabmod.LOWER_GHOST, out[lo][slabmod.LAST])
            unpack(sl, e, mu, parity, slabmod.UPPER_GHOST, out[hi][slabmod.FIRST])
    got = np.concatenate([interior(sl, e) for e, sl in zip(exts, slabs)])
    assert not np.array_equal(got, want)


# ------------------------------------------------------------ two gloo ranks
NS, NT, BETA, SEED, SWEEPS = 4, 8, 2.3, 7, 2


def _rank_main(rank, world, port, outdir):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ext = slabmod.slab_extent(NS, NT, rank, world)
        sl = slab_from(oracle.hot_start(NS, NT, SEED), ext)
        trials = np.zeros(8, dtype=np.int64)
        for s in range(SWEEPS):
            for mu, parity in slabmod.PHASES:
                trials[2 * mu + parity] += oracle.slab_phase(NS, NT, ext.t0, ext.nt_local, BETA, SEED, s, mu,
                                                             parity, sl)
                out = {side: torch.from_numpy(pack(sl, ext, mu, parity, side))
                       for side in (slabmod.FIRST, slabmod.LAST)}
                inn = {side: torch.empty_like(out[slabmod.FIRST])
                       for side in (slabmod.LOWER_GHOST, slabmod.UPPER_GHOST)}
                reqs = []
                for kind, peer, side, tag in slabmod.exchange_plan(rank, world):
                    if kind == "send":
                        reqs.append(dist.isend(out[side], peer, tag=tag))
                    else:
                        reqs.append(dist.irecv(inn[side], peer, tag=tag))
                for r in reqs:
                    r.wait()
                for side in (slabmod.LOWER_GHOST, slabmod.UPPER_GHOST):
                    unpack(sl, ext, mu, parity, side, inn[side].numpy())
        np.save(os.path.join(outdir, f"interior{rank}.npy"), interior(sl, ext))
        np.save(os.path.join(outdir, f"trials{rank}.npy"), trials)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_equal_the_lattice_chain():
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True)
        got = np.concatenate([np.load(os.path.join(d, f"interior{r}.npy")) for r in range(world)])
        trials = sum(np.load(os.path.join(d, f"trials{r}.npy")) for r in range(world))
    want, want_trials = full_chain(NS, NT, BETA, SEED, SWEEPS, False)
    assert np.array_equal(got, want)
    assert np.array_equal(trials, want_trials)
