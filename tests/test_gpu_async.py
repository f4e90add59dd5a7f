"""Asynchronous C-ABI forms (su2_set_links_async, su2_generate_async,
su2_get_links_async, su2_sync): the same chain as the synchronous calls and
as the oracle, bit for bit, also with several configurations in flight on
their own streams (the pipeline the end-to-end benchmark runs)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_1486_gb300 import su2

pytestmark = pytest.mark.gpu


def pinned(shape, dtype):
    return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()


def start_links(ns, nt, seed):
    return oracle.hot_start(ns, nt, seed)


@pytest.mark.parametrize("ns,nt,beta", [(8, 8, 2.3), (6, 4, 6.0)])
def test_async_step_equals_sync_step_and_oracle(ns, nt, beta):
    seed = 21
    x0 = start_links(ns, nt, 5)
    ref = x0.copy()
    oracle.heatbath_sweep(ns, nt, beta, seed, 0, ref)
    oracle.heatbath_sweep(ns, nt, beta, seed, 1, ref)
    p_ref = oracle.plaquette(ns, nt, ref)

    a = su2.su2_create(ns, nt, beta, seed, su2.SU2_COLD, stream=torch.cuda.Stream())
    b = su2.su2_create(ns, nt, beta, seed, su2.SU2_COLD, stream=torch.cuda.Stream())
    try:
        su2.su2_set_links(a, x0)
        p_sync, l_sync, _ = su2.su2_generate(a, 2, 1, 0)
        y_sync = su2.su2_get_links(a, ns, nt)

        xin = pinned(x0.shape, torch.float32)
        xin[...] = x0
        yout = pinned(x0.shape, torch.float32)
        plaq = pinned(2, torch.float64)
        poly = pinned(2, torch.float64)
        su2.su2_set_links_async(b, xin)
        su2.su2_generate_async(b, 2, 1, 0, plaq, poly)
        su2.su2_get_links_async(b, yout)
        su2.su2_sync(b)
        assert np.array_equal(yout.view(np.uint32), y_sync.view(np.uint32))
        assert np.array_equal(yout.view(np.uint32), ref.view(np.uint32))
        assert np.array_equal(plaq, p_sync) and np.array_equal(poly, l_sync)
        assert abs(plaq[1] - p_ref) <= 1e-6 * max(abs(p_ref), 0.05)
    finally:
        su2.su2_destroy(a)
        su2.su2_destroy(b)


def test_three_configurations_in_flight_equal_three_sequential_chains():
    ns, nt, beta, steps = 8, 4, 2.5, 4
    seeds = [31, 32, 33]
    starts = [start_links(ns, nt, 100 + i) for i in range(3)]

    # reference: each chain alone, synchronous calls, configuration through the host
    want = []
    for seed, x in zip(seeds, starts):
        h = su2.su2_create(ns, nt, beta, seed, su2.SU2_COLD)
        try:
            cur, plaqs = x.copy(), []
            for _ in range(steps):
                su2.su2_set_links(h, cur)
                p, _, _ = su2.su2_generate(h, 1, 1, 0)
                cur = su2.su2_get_links(h, ns, nt)
                plaqs.append(p[0])
            want.append((cur, plaqs))
        finally:
            su2.su2_destroy(h)

    # pipelined: round robin over three handles, each on its own stream
    hs = [su2.su2_create(ns, nt, beta, s, su2.SU2_COLD, stream=torch.cuda.Stream()) for s in seeds]
    try:
        bufs = []
        for x in starts:
            a, b = pinned(x.shape, torch.float32), pinned(x.shape, torch.float32)
            a[...] = x
            bufs.append([a, b])
        plaq = [pinned(steps, torch.float64) for _ in hs]
        for k in range(steps * 3):
            i, step = k % 3, k // 3
            h = hs[i]
            su2.su2_sync(h)  # this handle's previous step is done: its output is the next input
            if step > 0:
                bufs[i].reverse()
            su2.su2_set_links_async(h, bufs[i][0])
            su2.su2_generate_async(h, 1, 1, 0, plaq[i][step:step + 1], None)
            su2.su2_get_links_async(h, bufs[i][1])
        for h in hs:
            su2.su2_sync(h)
        for i in range(3):
            got = bufs[i][1]
            assert np.array_equal(got.view(np.uint32), want[i][0].view(np.uint32)), i
            assert np.array_equal(plaq[i], np.array(want[i][1])), i
    finally:
        for h in hs:
            su2.su2_destroy(h)


@pytest.mark.parametrize("use_stream", [True, False])
def test_async_with_pageable_buffers_and_the_default_stream(use_stream):
    """Pageable host memory (staged by the driver) and a lattice on the legacy
    default stream give the same chain as the synchronous calls."""
    ns, nt, beta, seed = 6, 4, 2.4, 9
    x0 = start_links(ns, nt, 3)
    a = su2.su2_create(ns, nt, beta, seed, su2.SU2_COLD)
    b = su2.su2_create(ns, nt, beta, seed, su2.SU2_COLD, stream=torch.cuda.Stream() if use_stream else None)
    try:
        su2.su2_set_links(a, x0)
        p_sync, _, _ = su2.su2_generate(a, 3, 1, 0)
        y_sync = su2.su2_get_links(a, ns, nt)
        xin = x0.copy()                       # ordinary numpy memory
        yout = np.empty_like(x0)
        plaq = np.zeros(3)
        su2.su2_set_links_async(b, xin)
        su2.su2_generate_async(b, 3, 1, 0, plaq, None)
        su2.su2_get_links_async(b, yout)
        su2.su2_sync(b)
        assert np.array_equal(yout.view(np.uint32), y_sync.view(np.uint32))
        assert np.array_equal(plaq, p_sync)
    finally:
        su2.su2_destroy(a)
        su2.su2_destroy(b)


def test_async_calls_check_their_arguments():
    h = su2.su2_create(4, 4, 2.0, 1, su2.SU2_COLD)
    try:
        with pytest.raises(ValueError):
            su2.su2_set_links_async(h, np.zeros((256, 4, 4), dtype=np.float64))
        with pytest.raises(su2.SU2Error):
            su2.su2_generate_async(h, -1, 1, 0)
        su2.su2_sync(h)
    finally:
        su2.su2_destroy(h)
