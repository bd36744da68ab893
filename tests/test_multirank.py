"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas only).
The job time is the slowest rank's and the value counts all ranks' cells."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms_local = 10.0 + 5.0 * rank          # rank 1 is slower
    ms, value = bench.combine_ranks(ms_local, cells=1000, steps=4, ws=ws)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value))


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 15.0
        assert value == pytest.approx(2 * 1000 * 4 / 0.015 / 1e6)


def test_single_rank_is_unchanged():
    import bench
    ms, value = bench.combine_ranks(8.0, cells=500, steps=2, ws=1)
    assert ms == 8.0 and value == pytest.approx(500 * 2 / 0.008 / 1e6)
