"""The multi-rank (one process per GPU) bookkeeping of bench.py, on the CPU with
the gloo backend and two ranks: slowest-rank time, summed voxels, whole-job
value. The path shards by independent batches, so no data collective exists."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, total, value = bench.aggregate_ranks(1.0 + rank, 1000 * (rank + 1), world, torch.device("cpu"))
    dist.barrier()
    q.put((rank, ms, total, value))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, total, value in res:
        assert ms == 2.0 and total == 3000 and abs(value - 3000 / 0.002) < 1e-6


def test_single_rank_aggregation():
    import bench

    ms, total, value = bench.aggregate_ranks(0.5, 100, 1, torch.device("cpu"))
    assert (ms, total) == (0.5, 100) and abs(value - 200000.0) < 1e-9
