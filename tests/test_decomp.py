"""Host logic of the domain decomposition (no GPU): slab partition, the halo
exchange plan, and the exchange loop and time-step all-reduce over two gloo
ranks, with plain arrays standing in for the packed cells."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1406_7416_gb300.decomp import (distributed_exchange, exchange_plan, global_min,
                                          slab_partition, slab_workload)


@pytest.mark.parametrize("n,parts,periodic", [(16, 2, True), (16, 2, False), (12, 3, True),
                                              (13, 4, False), (9, 1, True), (5, 2, True)])
def test_plan_fills_every_halo_cell_from_its_owner(n, parts, periodic):
    halo = 2
    slabs = slab_partition(n, parts, halo, periodic)
    assert sum(s.width for s in slabs) == n
    assert [s.own[0] for s in slabs] == sorted(s.own[0] for s in slabs)
    plan = exchange_plan(slabs, n) if parts > 1 else []
    filled = {s.index: set() for s in slabs}
    for t in plan:
        o, r = slabs[t.owner], slabs[t.receiver]
        assert t.owner_range[1] - t.owner_range[0] == t.receiver_range[1] - t.receiver_range[0]
        for lo_, lr in zip(range(*t.owner_range), range(*t.receiver_range)):
            # the owner's cell is one of its own, and the same global cell
            assert o.lo_halo <= lo_ < o.lo_halo + o.width
            assert o.global_index(lo_, n) == r.global_index(lr, n)
            filled[r.index].add(lr)
    for s in slabs:
        halo_cells = set(range(s.lo_halo)) | set(range(s.lo_halo + s.width, s.local_n))
        assert filled[s.index] == halo_cells
        if parts > 1:
            # halo layers on every side with a neighbour; none at a physical boundary
            assert s.lo_halo == (halo if (periodic or s.index > 0) else 0)
            assert s.hi_halo == (halo if (periodic or s.index < parts - 1) else 0)


def test_slabs_narrower_than_the_halo_are_refused():
    with pytest.raises(ValueError):
        slab_partition(5, 4, 2, True)


def test_slab_workload_keeps_the_physical_boundaries():
    w = dict(dim=2, ncell=(16, 8), x0=(-1.0, 0.0), dx=(0.125, 0.25), bc=(2, 3, 0, 0))
    slabs = slab_partition(16, 2, 2, periodic=False)
    lo = slab_workload(w, slabs[0], 0, 2)
    hi = slab_workload(w, slabs[1], 0, 2)
    assert lo["ncell"] == (10, 8) and hi["ncell"] == (10, 8)
    assert lo["bc"] == (2, 1, 0, 0) and hi["bc"] == (1, 3, 0, 0)
    assert lo["x0"] == (-1.0, 0.0) and hi["x0"] == (-1.0 + 6 * 0.125, 0.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, parts, periodic, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo")
    slabs = slab_partition(n, parts, 2, periodic)
    plan = exchange_plan(slabs, n)
    rank_of = [i % world for i in range(parts)]
    # the "global state": cell g carries a payload of 3 values derived from g
    G = np.stack([np.arange(n) * 10.0 + k for k in range(3)], axis=1)
    local = {}
    for s in slabs:
        if rank_of[s.index] != rank:
            continue
        L = np.full((s.local_n, 3), np.nan)
        own = range(s.lo_halo, s.lo_halo + s.width)
        L[list(own)] = G[s.own[0]:s.own[1]]
        local[s.index] = L

    def pack(tr):
        return torch.from_numpy(local[tr.owner][tr.owner_range[0]:tr.owner_range[1]].copy())

    def make_buffer(tr):
        return torch.empty((tr.receiver_range[1] - tr.receiver_range[0], 3), dtype=torch.float64)

    def unpack(tr, t):
        local[tr.receiver][tr.receiver_range[0]:tr.receiver_range[1]] = t.numpy()

    distributed_exchange(plan, rank_of, rank, pack, unpack, make_buffer, dist)
    ok = all(np.array_equal(L, G[[s.global_index(l, n) for l in range(s.local_n)]])
             for s in slabs if s.index in local for L in [local[s.index]])
    dt = global_min(0.25 + rank, dist)
    dist.destroy_process_group()
    out.put((rank, ok, dt))


@pytest.mark.parametrize("n,parts,periodic", [(16, 2, True), (14, 4, False)])
def test_exchange_over_two_gloo_ranks(n, parts, periodic):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n, parts, periodic, out))
             for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok, dt in res:
        assert ok, rank
        assert dt == 0.25            # the minimum over the ranks
