"""Slab decomposition and batch sharding on CPU ranks (gloo), with the FP64 oracle
as the per-slab compute.

Each rank holds one slab of the grid; before every RK stage it packs its G = R+3
boundary layers, exchanges them with its neighbours through decomp.halo_exchange
(the function the GPU path uses over NCCL), evaluates the oracle's RHS on its slab
plus the received halo layers, and applies the Shu-Osher stage combination.  The
slabs put back together must equal the oracle's single-domain step bitwise: every
face sees the same stencil values either way.  The common time step's rate maxima
go through decomp.allreduce_max_rates as int64 bit patterns."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1808_04960_gb300 import decomp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    from paper_1808_04960_gb300 import workloads as W
    if name == "vortex2d":
        return W.isentropic_vortex(40, ny=46), 2
    if name == "quadrant2d":
        return W.four_quadrant(36, seed=3, ny=41), 2
    if name == "sod1d":
        return W.sod_1d(67), 3
    if name == "smooth3d":
        return W.smooth_field((23, 10, 12), seed=2), 1
    raise KeyError(name)


def _rates(U, dx, gamma):
    """max over cells of (|u_d| + c)/dx_d per direction (x, y, z), zero for absent ones."""
    from paper_1808_04960_gb300 import workloads as W
    rho, vel, p = W.primitive(U, gamma)
    c = np.sqrt(gamma * p / rho)
    out = np.zeros(3)
    for d, v in enumerate(vel):
        out[d] = np.max((np.abs(v) + c) / dx[d])
    return out


def _slab_step(U, o, slab, dt, ghost):
    """One SSP-RK3 step of this rank's slab (rows of U) with a halo exchange before each stage."""
    G = ghost
    rest = U.shape[2:]
    send = [torch.zeros((U.shape[0], G) + rest, dtype=torch.float64) for _ in range(2)]
    recv = [torch.zeros_like(send[0]) for _ in range(2)]

    def rhs(V):
        send[0].copy_(torch.from_numpy(np.ascontiguousarray(V[:, :G])))
        send[1].copy_(torch.from_numpy(np.ascontiguousarray(V[:, -G:])))
        decomp.halo_exchange(send[0], send[1], recv[0], recv[1], slab.lo_rank, slab.hi_rank)
        parts, off = [], 0
        if slab.lo_rank is not None:
            parts.append(recv[0].numpy())
            off = G
        parts.append(V)
        if slab.hi_rank is not None:
            parts.append(recv[1].numpy())
        Wd = np.ascontiguousarray(np.concatenate(parts, axis=1))
        L = o(Wd.shape[1:]).rhs(Wd)
        return L[:, off:off + V.shape[1]]

    # the oracle's Shu-Osher combination, operation for operation
    L = rhs(U)
    U1 = U + dt * L
    L = rhs(U1)
    U2 = 0.75 * U + 0.25 * (U1 + dt * L)
    L = rhs(U2)
    return U / 3.0 + 2.0 / 3.0 * (U2 + dt * L)


def _rank(rank, ws, port, name, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        (U0, meta), R = _case(name)
        G = R + 3
        gamma = meta.get("gamma", 1.4)
        shape = U0.shape[1:]
        slab = decomp.Slab(shape, meta["bc"], rank, ws, G)
        d = len(shape) - 1
        # the window's slab-axis boundary: the grid's own condition on an outer side; on a cut side
        # the window carries the G halo layers, so its boundary condition there never reaches the slab
        wbc = list(meta["bc"])
        wbc[d] = tuple("outflow" if b == "external" else b for b in slab.local_bc[d])
        ora = lambda wshape: oracle.Oracle(wshape, meta["dx"], tuple(wbc), R=R, ell_over_dx=12.0, gamma=gamma)
        full = oracle.Oracle(shape, meta["dx"], meta["bc"], R=R, ell_over_dx=12.0, gamma=gamma)
        # common time step from the ranks' rate maxima (int64 bit patterns, max-reduced)
        mine = _rates(U0[(slice(None), slab.rows)], meta["dx"], gamma)
        rates = torch.from_numpy(mine.view(np.int64).copy())
        decomp.allreduce_max_rates(rates)
        glob = rates.numpy().view(np.float64)
        dt = 0.4 / glob[:len(shape)].sum()
        ref_dt = full.cfl_dt(U0, 0.4)
        U = np.ascontiguousarray(U0[(slice(None), slab.rows)])
        for _ in range(2):
            U = _slab_step(U, ora, slab, dt, G)
        ref = full.run(U0, dt, 2)[(slice(None), slab.rows)]
        out[rank] = (float(np.abs(U - ref).max()), bool(np.array_equal(U, ref)), abs(dt - ref_dt) / ref_dt,
                     slab.lo_rank, slab.hi_rank)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,ws", [("vortex2d", 2), ("vortex2d", 3), ("quadrant2d", 2), ("sod1d", 2),
                                     ("smooth3d", 2)])
def test_slabs_match_single_domain_oracle(name, ws):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, name, out), nprocs=ws, join=True)
        res = dict(out)
    assert sorted(res) == list(range(ws))
    for r, (err, exact, dt_rel, lo, hi) in res.items():
        assert exact, (name, r, err)
        assert dt_rel < 1e-15, (name, r, dt_rel)


def test_partition_and_neighbours():
    parts = decomp.slab_partition(10, 3, 2)
    assert parts == [(0, 4), (4, 3), (7, 3)]
    assert sum(c for _, c in parts) == 10
    with pytest.raises(ValueError):
        decomp.slab_partition(10, 3, 5)            # a slab would hold fewer than G cells
    per = (("periodic", "periodic"), ("periodic", "periodic"))
    out = (("outflow", "outflow"), ("outflow", "outflow"))
    s = [decomp.Slab((10, 8), per, r, 3, 2) for r in range(3)]
    assert [(x.lo_rank, x.hi_rank) for x in s] == [(2, 1), (0, 2), (1, 0)]
    assert all(x.local_bc[1] == ("external", "external") and x.local_bc[0] == per[0] for x in s)
    t = [decomp.Slab((10, 8), out, r, 3, 2) for r in range(3)]
    assert [(x.lo_rank, x.hi_rank) for x in t] == [(None, 1), (0, 2), (1, None)]
    assert [x.local_bc[1] for x in t] == [("outflow", "external"), ("external", "external"),
                                          ("external", "outflow")]
    one = decomp.Slab((10, 8), per, 0, 1, 2)
    assert (one.lo_rank, one.hi_rank, one.local_bc) == (None, None, per)
    assert t[1].halo_rows(0) == [2, 3] and t[1].halo_rows(1) == [7, 8]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_instances_cover_and_balance(world):
    rng = np.random.default_rng(5)
    insts = [(int(rng.integers(64, 1025)), int(rng.integers(64, 1025)), int(rng.integers(1, 4))) for _ in range(256)]
    costs = [decomp.instance_cost(nx, ny, R) for nx, ny, R in insts]
    parts, loads = decomp.shard_instances(costs, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))                      # every instance exactly once
    assert all(p == sorted(p) for p in parts)
    for p, load in zip(parts, loads):
        assert abs(sum(costs[i] for i in p) - load) < 1e-6 * load
    assert max(loads) - sum(costs) / world < max(costs)         # greedy bound


def _rank_leaves(rank, ws, port, out):
    """Rank 1 leaves between steps (after the first exchange, before the second) without
    tearing down its process group; rank 0's next exchange must end in an error, not a hang."""
    import datetime
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=datetime.timedelta(seconds=10))
    G, shape = 5, (4, 12, 8)
    send = [torch.full((shape[0], G, shape[2]), float(rank)) for _ in range(2)]
    recv = [torch.zeros((shape[0], G, shape[2])) for _ in range(2)]
    lo = hi = 1 - rank                       # two ranks on a periodic ring
    decomp.halo_exchange(send[0], send[1], recv[0], recv[1], lo, hi)
    out[(rank, "first")] = float(recv[0][0, 0, 0])
    if rank == 1:
        os._exit(0)                          # leaves without a word, none of its work in flight
    t0 = time.time()
    try:
        decomp.halo_exchange(send[0], send[1], recv[0], recv[1], lo, hi)
        out[(rank, "second")] = "completed"
    except Exception as e:                   # noqa: BLE001 - the transport's own error type
        out[(rank, "second")] = f"error: {type(e).__name__}"
    out[(rank, "seconds")] = time.time() - t0
    os._exit(0)


def test_exchange_with_a_departed_rank_fails_on_the_host():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with mp.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_leaves, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(60)
        alive = [p.is_alive() for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        res = dict(out)
    assert not any(alive), "a rank hung"
    assert res[(0, "first")] == 1.0 and res[(1, "first")] == 0.0
    assert str(res[(0, "second")]).startswith("error"), res
    assert res[(0, "seconds")] < 30
