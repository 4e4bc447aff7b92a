"""Multi-rank host logic: slab decomposition of one grid and instance sharding of a batch.

Slabs.  One grid is cut along its slowest axis (x in 1D, y in 2D, z in 3D) into
one slab per rank; neighbouring slabs exchange G = R+3 boundary layers before
every RK stage (the corrected flux of Eq. numFlux_cor differenced by Eq.
disc_fd reaches G cells), and a common CFL time step takes one max-reduction
of the three per-direction wavespeed maxima per step.  The paper's solver is
parallelized the same way across CPU cores (Section 5; its vortex timings of
Section 6.2 ran on four cores); here each slab is one GPU and the transport is
torch.distributed (NCCL on GPUs, gloo on CPU tensors).  The cut sides of a slab
are GPWENO_BC_EXTERNAL sides of its plan; the outer sides keep the grid's
boundary condition (periodic grids close the ring of slabs).

Batches.  Independent instances are split over ranks by estimated cost, with
no exchange at all.
"""
from __future__ import annotations

from dataclasses import dataclass

# message tags: a slab's top layers travel up (to the next slab's low halo),
# its bottom layers travel down (to the previous slab's high halo)
TAG_UP, TAG_DOWN = 11, 12


def slab_partition(n: int, world: int, ghost: int):
    """(start, count) of `world` slabs of an axis of n cells; counts differ by at most one
    (the first n % world slabs take one more).  Every slab must hold at least `ghost` cells,
    so that its halo comes from its direct neighbours only."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(n, world)
    parts, start = [], 0
    for r in range(world):
        cnt = base + (1 if r < extra else 0)
        parts.append((start, cnt))
        start += cnt
    if world > 1 and min(c for _, c in parts) < ghost:
        raise ValueError(f"{n} cells over {world} slabs leaves fewer than G = {ghost} cells in a slab")
    return parts


@dataclass
class Slab:
    """Rank `rank`'s slab of a grid of array shape `shape` ((nx,), (ny, nx) or (nz, ny, nx))
    with boundary conditions `bc` ((lo, hi) pairs in (x, y, z) order)."""
    shape: tuple
    bc: tuple
    rank: int
    world: int
    ghost: int

    def __post_init__(self):
        self.shape = tuple(int(s) for s in self.shape)
        self.ndim = len(self.shape)
        d = self.ndim - 1                          # slab dimension in (x, y, z) order = array axis 0
        self.start, self.count = slab_partition(self.shape[0], self.world, self.ghost)[self.rank]
        periodic = self.bc[d][0] == "periodic"
        if self.world == 1:
            self.lo_rank = self.hi_rank = None
        else:
            self.lo_rank = self.rank - 1 if self.rank > 0 else (self.world - 1 if periodic else None)
            self.hi_rank = self.rank + 1 if self.rank < self.world - 1 else (0 if periodic else None)
        bc = [tuple(b) for b in self.bc]
        if self.world > 1:
            lo = "external" if self.lo_rank is not None else bc[d][0]
            hi = "external" if self.hi_rank is not None else bc[d][1]
            bc[d] = (lo, hi)
        self.local_bc = tuple(bc)
        self.local_shape = (self.count,) + self.shape[1:]

    @property
    def rows(self):
        """Slice of the slab along array axis 0 of the whole grid."""
        return slice(self.start, self.start + self.count)

    def halo_rows(self, side):
        """Global indices (along array axis 0, before any periodic wrap) of the G layers of the
        low (side 0) or high (side 1) halo, in increasing order."""
        if side == 0:
            return list(range(self.start - self.ghost, self.start))
        return list(range(self.start + self.count, self.start + self.count + self.ghost))


def halo_exchange(send_lo, send_hi, recv_lo, recv_hi, lo_rank, hi_rank, group=None):
    """Send this slab's bottom layers down and its top layers up; receive the lower neighbour's
    top layers into recv_lo and the upper neighbour's bottom layers into recv_hi.

    Sends are issued in the order (up, down) and receives in the order (from below, from
    above), so that with two ranks on a periodic ring -- where both neighbours are the same
    rank -- the two messages of a pair land in the right buffers whether the transport matches
    by tag (gloo) or by issue order (NCCL)."""
    import torch.distributed as dist
    ops = []
    if hi_rank is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, hi_rank, group, TAG_UP))
    if lo_rank is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, lo_rank, group, TAG_DOWN))
    if lo_rank is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, lo_rank, group, TAG_UP))
    if hi_rank is not None:
        ops.append(dist.P2POp(dist.irecv, recv_hi, hi_rank, group, TAG_DOWN))
    if not ops:
        return
    if dist.get_backend(group) == "nccl":
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    else:
        reqs = [op.op(op.tensor, op.peer, op.group, op.tag) for op in ops]
        for req in reqs:
            req.wait()


def allreduce_max_rates(rates, group=None):
    """Max-reduce the exported rate maxima over the ranks (int64 bit patterns of non-negative
    doubles order like the doubles)."""
    import torch.distributed as dist
    dist.all_reduce(rates, op=dist.ReduceOp.MAX, group=group)


class SlabStepper:
    """SSP-RK3 steps of one rank's slab through the C ABI, halo exchange before each stage.

    plan: the slab's gpweno Plan (local shape, local boundary conditions of `slab`);
    exchange: callable(send_lo, send_hi, recv_lo, recv_hi) that moves the halo layers
    (defaults to halo_exchange with the slab's neighbours over torch.distributed)."""

    def __init__(self, plan, slab: Slab, exchange=None, group=None):
        import torch
        self.plan, self.slab = plan, slab
        self.scratch = plan.new_scratch()
        ext = slab.lo_rank is not None or slab.hi_rank is not None
        self.ext = ext
        if ext:
            self.send = [plan.new_halo(), plan.new_halo()]
            self.recv = [plan.new_halo(), plan.new_halo()]
            plan.set_halo(self.recv[0] if slab.lo_rank is not None else None,
                          self.recv[1] if slab.hi_rank is not None else None)
        self.rates = torch.zeros(3, dtype=torch.int64, device="cuda")
        self.group = group
        self.exchange = exchange or (lambda sl, sh, rl, rh: halo_exchange(sl, sh, rl, rh, slab.lo_rank,
                                                                           slab.hi_rank, group))

    def pack(self, k, U, stream=None):
        if self.ext:
            self.plan.halo_pack(self.plan.stage_input(k, U, self.scratch), self.send[0], self.send[1], stream)

    def stage(self, k, U, dt=0.0, dt_dev=None, stream=None):
        self.plan.rk3_stage(k, U, self.scratch, dt=dt, dt_dev=dt_dev, stream=stream)

    def step(self, U, dt=0.0, dt_dev=None, stream=None):
        if not self.ext:
            self.plan.rk3_step(U, self.scratch, dt=dt, dt_dev=dt_dev, stream=stream)
            return
        for k in range(3):
            self.pack(k, U, stream)
            self.exchange(self.send[0], self.send[1], self.recv[0], self.recv[1])
            self.stage(k, U, dt, dt_dev, stream)
        if dt_dev is not None and self.plan.cfl > 0:
            self.plan.rate_export(self.rates, stream)
            allreduce_max_rates(self.rates, self.group)
            self.plan.dt_from_rates(self.rates, self.plan.cfl, dt_dev, stream)


def shard_instances(costs, world: int):
    """Split instances with estimated costs over `world` ranks: longest first to the least
    loaded rank (ties to the lowest rank), each rank's list in increasing instance order.
    Every instance goes to exactly one rank; the largest load exceeds the mean by less than
    the largest single cost."""
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts], loads


def instance_cost(nx: int, ny: int, R: int) -> float:
    """Estimated stage cost of a 2D instance: cells x operations per cell-stage."""
    from . import costmodel
    return float(nx) * float(ny) * costmodel.flops_per_cell_stage(R, 2)
