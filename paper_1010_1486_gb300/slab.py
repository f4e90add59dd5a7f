"""Time-slab decomposition of one lattice over ranks (Sec. 4, multi-GPU part,
and Fig. 1 of Cardoso & Bicudo, LAT2010).

Rank r of W holds the time slices t0 = r Nt/W ... t0 + Nt/W - 1 of an
Ns^3 x Nt lattice plus one ghost slice on each side (Ns^3 x (Nt/W + 2) sites).
A sweep is the lattice's eight phases (mu = 0..3, even then odd sites); every
rank runs each phase on its interior, then the links that phase changed in the
boundary slices -- U_mu of that parity in the first and the last interior
slice, Ns^3 / 2 links each -- move to the neighbours' ghost slices before the
next phase reads them.  The random numbers of a link are keyed by its global
site, so the decomposed chain is the single lattice's chain bit for bit.

The paper moved the border cells through host memory with an OpenMP barrier
between the GPUs' threads; here the ranks are processes and the transport is
``torch.distributed`` point-to-point messages (gloo with host buffers, or NCCL
with device buffers).  The library packs and unpacks the boundary slices
(``su2_slab_pack`` / ``su2_slab_unpack``); this module only sequences phases
and messages.  Slabs in one process exchange with ``su2_slab_exchange``
instead (:class:`LocalSlabs`).
"""
from __future__ import annotations

from dataclasses import dataclass

# message tags: what the receiver does with the slice
TAG_TO_UPPER_GHOST = 1   # the sender's first interior slice (the receiver is the lower neighbour)
TAG_TO_LOWER_GHOST = 2   # the sender's last interior slice (the receiver is the upper neighbour)

# su2_slab_pack sides and su2_slab_unpack sides
FIRST, LAST = 0, 1            # interior slices that leave
LOWER_GHOST, UPPER_GHOST = 0, 1  # ghost slices that are filled

PHASES = tuple((mu, parity) for mu in range(4) for parity in range(2))


@dataclass(frozen=True)
class SlabExtent:
    """The time slices of one rank: local slice tl holds global slice
    (t0 - 1 + tl) mod nt, tl = 0 and nt_local + 1 are the ghosts."""
    ns: int
    nt: int
    t0: int
    nt_local: int


def slab_extent(ns: int, nt: int, rank: int, world: int) -> SlabExtent:
    """Equal slabs; each must hold an even number (>= 2) of slices so that the
    even/odd split of every slab matches the lattice's."""
    if world < 1 or nt % world:
        raise ValueError(f"Nt = {nt} does not split into {world} equal slabs")
    ntl = nt // world
    if ntl < 2 or ntl % 2:
        raise ValueError(f"a slab of {ntl} slices: slabs need an even number >= 2")
    return SlabExtent(ns, nt, rank * ntl, ntl)


def neighbours(rank: int, world: int) -> tuple[int, int]:
    """(lower, upper) neighbour ranks on the periodic time axis."""
    return (rank - 1) % world, (rank + 1) % world


def exchange_plan(rank: int, world: int):
    """What follows every phase on this rank, as (kind, peer, side, tag):
    the first interior slice goes to the lower neighbour's upper ghost, the
    last to the upper neighbour's lower ghost; the lower ghost comes from the
    lower neighbour's last slice, the upper ghost from the upper neighbour's
    first.  With one rank the slab is its own neighbour on both sides."""
    lo, hi = neighbours(rank, world)
    return (("send", lo, FIRST, TAG_TO_UPPER_GHOST),
            ("send", hi, LAST, TAG_TO_LOWER_GHOST),
            ("recv", lo, LOWER_GHOST, TAG_TO_LOWER_GHOST),
            ("recv", hi, UPPER_GHOST, TAG_TO_UPPER_GHOST))


class DistributedSlab:
    """One rank's slab in a process group: ``sweep(n)`` runs n sweeps with the
    boundary exchange after every phase.  ``device_buffers`` keeps the
    messages in device memory (for NCCL); otherwise they go through pinned
    host memory (gloo), as the paper's host-staged exchange did."""

    def __init__(self, ns: int, nt: int, beta: float, seed: int, start: int, group=None, stream=None,
                 device_buffers: bool = False):
        import torch
        import torch.distributed as dist

        from . import su2

        self.su2, self.dist, self.torch = su2, dist, torch
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.extent = slab_extent(ns, nt, self.rank, self.world)
        self.h = su2.su2_slab_create(ns, nt, self.extent.t0, self.extent.nt_local, beta, seed, start, stream)
        nbytes = su2.su2_slab_boundary_bytes(self.h)
        dev = torch.device("cuda", torch.cuda.current_device()) if device_buffers else None
        kw = dict(dtype=torch.uint8, device=dev) if device_buffers else dict(dtype=torch.uint8, pin_memory=True)
        self.out = [torch.empty(nbytes, **kw) for _ in range(2)]
        self.inn = [torch.empty(nbytes, **kw) for _ in range(2)]
        self.on_device = device_buffers

    def close(self):
        if self.h:
            self.su2.su2_slab_destroy(self.h)
            self.h = None

    def set_sampler(self, sampler: int):
        self.su2.su2_slab_set_sampler(self.h, sampler)

    def _exchange(self, mu: int, parity: int):
        su2 = self.su2
        for side in (FIRST, LAST):
            su2.su2_slab_pack(self.h, mu, parity, side, self.out[side].data_ptr())
        su2.su2_slab_sync(self.h)
        if self.world == 1:
            su2.su2_slab_unpack(self.h, mu, parity, UPPER_GHOST, self.out[FIRST].data_ptr())
            su2.su2_slab_unpack(self.h, mu, parity, LOWER_GHOST, self.out[LAST].data_ptr())
            su2.su2_slab_sync(self.h)
            return
        reqs = []
        for kind, peer, side, tag in exchange_plan(self.rank, self.world):
            if kind == "send":
                reqs.append(self.dist.isend(self.out[side], peer, group=self.group, tag=tag))
            else:
                reqs.append(self.dist.irecv(self.inn[side], peer, group=self.group, tag=tag))
        for r in reqs:
            r.wait()
        for side in (LOWER_GHOST, UPPER_GHOST):
            su2.su2_slab_unpack(self.h, mu, parity, side, self.inn[side].data_ptr())
        su2.su2_slab_sync(self.h)

    def sweep(self, n: int = 1):
        for _ in range(n):
            for mu, parity in PHASES:
                self.su2.su2_slab_phase(self.h, mu, parity)
                self._exchange(mu, parity)


class LocalSlabs:
    """All slabs of a lattice in one process (on one device or several):
    phases slab by slab, boundary exchange by device copies."""

    def __init__(self, ns: int, nt: int, nslabs: int, beta: float, seed: int, start: int, streams=None):
        from . import su2

        self.su2 = su2
        self.extents = [slab_extent(ns, nt, r, nslabs) for r in range(nslabs)]
        streams = streams or [None] * nslabs
        self.h = [su2.su2_slab_create(ns, nt, e.t0, e.nt_local, beta, seed, start, s)
                  for e, s in zip(self.extents, streams)]

    def close(self):
        for h in self.h:
            self.su2.su2_slab_destroy(h)
        self.h = []

    def set_sampler(self, sampler: int):
        for h in self.h:
            self.su2.su2_slab_set_sampler(h, sampler)

    def sweep(self, n: int = 1):
        k = len(self.h)
        for _ in range(n):
            for mu, parity in PHASES:
                for h in self.h:
                    self.su2.su2_slab_phase(h, mu, parity)
                for r in range(k):
                    self.su2.su2_slab_exchange(self.h[r], self.h[(r + 1) % k], mu, parity)
        for h in self.h:
            self.su2.su2_slab_sync(h)
