"""Domain decomposition of one grid into slabs along one axis.

The paper runs its largest problems on many processes, each owning a block of
the grid (Sec. 5.8), and the flux correction of Sec. 4.4 couples the cells on
both sides of a block edge.  Here each slab is an ordinary libadg state whose
grid holds the slab's own cells plus `halo` layers of the neighbouring slabs'
cells on each side that has a neighbour.  Before every step the halo layers
are refilled from their owners (adg_pack_cells / adg_unpack_cells: DOFs,
flags, stored subcell data and the per-cell extrema of the subcell data),
the time step is the minimum of the slabs' CFL steps (an all-reduce across
ranks), and every slab takes the same step.  One step reads the level-n data
of the cells within two cells of an owned cell (the face neighbours' traces
and detector bounds, and the troubled status and sub-face fluxes of the
neighbours that feed the flux correction), so with two halo layers the owned
cells' new level equals that of the undivided grid bit for bit; the halo
cells' own results are overwritten by the next exchange.

Host logic only: the partition, the exchange plan and the exchange loop,
which runs all slabs in one process (one GPU) or one slab per rank over
torch.distributed (NCCL between GPUs, gloo on the CPU).  The arithmetic of the
step stays in libadg.
"""
from dataclasses import dataclass

import numpy as np

HALO = 2
TRANSMISSIVE = 1
PERIODIC = 0


@dataclass
class Slab:
    index: int
    own: tuple          # global owned range [a, b) along the split axis
    lo_halo: int        # halo layers below / above (0 at a physical boundary)
    hi_halo: int

    @property
    def width(self):
        return self.own[1] - self.own[0]

    @property
    def local_n(self):
        return self.lo_halo + self.width + self.hi_halo

    def global_index(self, l, n):
        """Global index along the split axis of local index l (wrapped)."""
        return (self.own[0] - self.lo_halo + l) % n


@dataclass
class Transfer:
    owner: int          # slab that owns the cells
    owner_range: tuple  # local range [a, b) along the split axis in the owner's grid
    receiver: int
    receiver_range: tuple


def slab_partition(n, parts, halo=HALO, periodic=False):
    """`parts` slabs of nearly equal width covering n cells, with `halo`
    layers on every side that has a neighbour (both sides when periodic)."""
    if parts < 1 or parts > n:
        raise ValueError("need 1 <= parts <= cells along the axis")
    bounds = [n * p // parts for p in range(parts + 1)]
    slabs = []
    for p in range(parts):
        a, b = bounds[p], bounds[p + 1]
        if parts > 1 and b - a < halo:
            raise ValueError(f"slab {p} is {b - a} cells wide, narrower than the halo ({halo})")
        lo = halo if (parts > 1 and (periodic or p > 0)) else 0
        hi = halo if (parts > 1 and (periodic or p < parts - 1)) else 0
        slabs.append(Slab(p, (a, b), lo, hi))
    return slabs


def exchange_plan(slabs, n):
    """Transfers that refill every halo from the slab owning its cells."""
    owner_of = np.empty(n, dtype=int)
    for s in slabs:
        owner_of[s.own[0]:s.own[1]] = s.index
    plan = []
    for r in slabs:
        for lo_l, hi_l in ((0, r.lo_halo), (r.lo_halo + r.width, r.local_n)):
            if hi_l <= lo_l:
                continue
            g = [r.global_index(l, n) for l in range(lo_l, hi_l)]
            o = slabs[owner_of[g[0]]]
            if any(owner_of[x] != o.index for x in g):
                raise ValueError("a halo spans two owners: slabs narrower than the halo")
            lo_o = (g[0] - o.own[0]) % n + o.lo_halo
            plan.append(Transfer(o.index, (lo_o, lo_o + len(g)), r.index, (lo_l, hi_l)))
    return plan


def slab_workload(w, slab, axis, parts):
    """The workload dict of one slab's local grid: its cells along `axis`
    from the first halo layer on, transmissive on sides with a halo (those
    cells are refilled before every step) and the global boundary kinds
    elsewhere."""
    loc = dict(w)
    n = list(w["ncell"])
    n[axis] = slab.local_n
    loc["ncell"] = tuple(n)
    x0 = list(w["x0"])
    x0[axis] = w["x0"][axis] + (slab.own[0] - slab.lo_halo) * w["dx"][axis]
    loc["x0"] = tuple(x0)
    bc = list(w["bc"])
    if parts > 1:
        if slab.lo_halo:
            bc[2 * axis] = TRANSMISSIVE
        if slab.hi_halo:
            bc[2 * axis + 1] = TRANSMISSIVE
    loc["bc"] = tuple(bc)
    return loc


def _axis_take(a, idx, axis, dim):
    """Cells `idx` along grid axis `axis` of a [cell][...] array (ABI order,
    x fastest) of a grid with cell counts `dim`."""
    shp = tuple(dim[::-1]) + a.shape[1:]
    A = a.reshape(shp)
    ax = len(dim) - 1 - axis
    B = np.take(A, idx, axis=ax)
    return B.reshape((-1,) + a.shape[1:])


def _axis_put(dst, dst_dim, src, src_dim, dst_idx, src_idx, axis):
    D = dst.reshape(tuple(dst_dim[::-1]) + dst.shape[1:])
    S = src.reshape(tuple(src_dim[::-1]) + src.shape[1:])
    ax = len(dst_dim) - 1 - axis
    sl_d = [slice(None)] * D.ndim
    sl_s = [slice(None)] * S.ndim
    sl_d[ax] = dst_idx
    sl_s[ax] = src_idx
    D[tuple(sl_d)] = S[tuple(sl_s)]


class Decomposed:
    """One grid as `parts` slab states along `axis` in this process.

    The slabs share the solvers' stream (libadg's default), so the exchange's
    pack, unpack and the steps are ordered on it.  Buffers of the packed
    cells are device tensors from torch."""

    def __init__(self, w, parts, axis=0, halo=HALO, prec=0):
        from . import adg
        self.w, self.axis, self.parts = w, axis, parts
        self.dim = w["dim"]
        self.n = w["ncell"][axis]
        periodic = w["bc"][2 * axis] == PERIODIC
        self.slabs = slab_partition(self.n, parts, halo, periodic)
        self.plan = exchange_plan(self.slabs, self.n) if parts > 1 else []
        self.solvers = [adg.Solver.from_workload(slab_workload(w, s, axis, parts), prec)
                        for s in self.slabs]
        self._bufs = {}

    # -- data in and out -----------------------------------------------------
    def _local_dims(self, s):
        d = list(self.w["ncell"])
        d[self.axis] = s.local_n
        return d

    def load_full(self, dofs, beta, sub):
        """Each slab takes its cells (halo layers included) of the global
        state (host arrays in the ABI layout)."""
        for s, sol in zip(self.slabs, self.solvers):
            idx = [s.global_index(l, self.n) for l in range(s.local_n)]
            g = self.w["ncell"]
            sol.load_full(_axis_take(dofs, idx, self.axis, g), _axis_take(beta, idx, self.axis, g),
                          _axis_take(sub, idx, self.axis, g))

    def read_full(self):
        """The global state assembled from the slabs' own cells."""
        parts = [sol.read_full() for sol in self.solvers]
        cells = int(np.prod(self.w["ncell"]))
        out = [np.empty((cells,) + a.shape[1:], dtype=a.dtype) for a in parts[0]]
        for s, arrs in zip(self.slabs, parts):
            own_local = list(range(s.lo_halo, s.lo_halo + s.width))
            own_global = list(range(s.own[0], s.own[1]))
            for dst, src in zip(out, arrs):
                _axis_put(dst, self.w["ncell"], src, self._local_dims(s), own_global, own_local,
                          self.axis)
        return tuple(out)

    # -- stepping ------------------------------------------------------------
    def _box(self, slab, rng):
        lo = [0] * self.dim
        hi = list(self._local_dims(slab))
        lo[self.axis], hi[self.axis] = rng
        return lo, hi

    def _buffer(self, key, nbytes):
        import torch
        b = self._bufs.get(key)
        if b is None or b.numel() < nbytes:
            b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            self._bufs[key] = b
        return b

    def exchange(self):
        """Refill every halo from its owner, device to device."""
        for t, tr in enumerate(self.plan):
            o, r = self.slabs[tr.owner], self.slabs[tr.receiver]
            lo_o, hi_o = self._box(o, tr.owner_range)
            lo_r, hi_r = self._box(r, tr.receiver_range)
            count = int(np.prod(np.array(hi_o) - np.array(lo_o)))
            buf = self._buffer(t, self.solvers[tr.owner].halo_bytes(count))
            self.solvers[tr.owner].pack_cells(lo_o, hi_o, buf.data_ptr())
            self.solvers[tr.receiver].unpack_cells(lo_r, hi_r, buf.data_ptr())

    def max_dt(self, cfl):
        """Eq. (cfl) over the whole grid: the minimum of the slabs' steps
        (after an exchange every slab sees exact data)."""
        return min(sol.max_dt(cfl) for sol in self.solvers)

    def step(self, dt):
        self.exchange()
        for sol in self.solvers:
            sol.step(dt)

    def step_cfl(self, cfl):
        self.exchange()
        dt = self.max_dt(cfl)
        for sol in self.solvers:
            sol.step(dt)
        return dt

    def status(self):
        return [sol.status() for sol in self.solvers]

    def close(self):
        for sol in self.solvers:
            sol.close()
        self._bufs = {}


def distributed_exchange(plan, rank_of, rank, pack, unpack, make_buffer, comm):
    """One halo exchange with the slabs spread over ranks (slab i on rank
    rank_of[i]).  pack(transfer) returns the owner's packed tensor,
    make_buffer(transfer) an empty tensor of the same size for the receiver,
    unpack(transfer, tensor) stores it; comm is torch.distributed.  Transfers
    between slabs of one rank are copied directly."""
    reqs, pending = [], []
    for t, tr in enumerate(plan):
        o_rank, r_rank = rank_of[tr.owner], rank_of[tr.receiver]
        if o_rank == rank and r_rank == rank:
            unpack(tr, pack(tr))
        elif o_rank == rank:
            reqs.append(comm.isend(pack(tr), dst=r_rank, tag=t))
        elif r_rank == rank:
            buf = make_buffer(tr)
            reqs.append(comm.irecv(buf, src=o_rank, tag=t))
            pending.append((tr, buf))
    for q in reqs:
        q.wait()
    for tr, buf in pending:
        unpack(tr, buf)


def global_min(x, comm, device=None):
    """The minimum of a scalar over all ranks (the time step's all-reduce)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    comm.all_reduce(t, op=comm.ReduceOp.MIN)
    return float(t.item())
