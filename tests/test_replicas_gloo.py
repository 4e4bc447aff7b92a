"""The multi-rank host logic of bench.py on CPU: two gloo ranks (the GPU runs use one
process per GPU over NCCL with the same code).  Each rank times its own replica; the
job's time is the slowest rank's, taken after a barrier on both sides."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        bench.barrier(ws)
        out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, ws)
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
