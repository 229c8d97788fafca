"""The N>1 bench path: independent replicas, the job's time is the slowest
rank's and its work the sum over ranks (world size 2, gloo on CPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 250.0][rank]
    cells = [1000, 3000][rank]
    value, ms_max = bench.combine_ranks(ms, cells, steps=10)
    q.put((rank, value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max in out:
        assert ms_max == 250.0
        assert value == pytest.approx(4000 * 10 / 0.25)


def test_combine_ranks_single_process():
    import bench
    v, ms = bench.combine_ranks(200.0, 500, 4)
    assert ms == 200.0 and v == pytest.approx(500 * 4 / 0.2)
