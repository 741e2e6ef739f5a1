"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica, combine into one whole-job number (max time over ranks)."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = [2.0, 5.0][rank]        # rank 1 is the slow one
    t_max, value = bench.combine_ranks(t_local, steps=3, world=world, dist=dist,
                                       device=torch.device("cpu"))
    q.put((rank, t_max, value))
    dist.destroy_process_group()


def test_two_rank_max_time_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, value in out:
        assert t_max == 5.0                 # the slowest rank sets the time
        assert value == pytest.approx(2 * 3 / 5.0)   # all ranks' solves / that time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.combine_ranks(2.0, 4, 1) == (2.0, 2.0)
