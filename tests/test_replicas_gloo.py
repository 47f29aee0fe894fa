"""Multi-process host logic of the benchmark on CPU (gloo, world size 2).

Each rank runs its own replica of the workload; the whole-job figure is the
units all ranks processed over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [120.0, 150.0][rank]
    units = [1.0e9, 1.0e9 + 7][rank]
    t, u = bench.combine_ranks(ms, units, dist, "cpu")
    q.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_max_time_sum_units():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u in got:
        assert t == 150.0
        assert u == pytest.approx(2.0e9 + 7)


def test_combine_ranks_single_process_is_identity():
    import bench

    assert bench.combine_ranks(3.0, 5.0) == (3.0, 5.0)
