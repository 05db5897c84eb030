"""The multi-process path of bench.py on the CPU: two gloo ranks.

On N GPUs bench.py runs N independent replicas of the workload (the method
shards by subtrees with an exchange per upper stage, but every run here has one
GPU, so no collective is written); the ranks meet only at the barriers around
the timed region and in the reduction that makes the job's time its slowest
rank's.  This test runs that reduction and the barrier in two gloo processes.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        dist.barrier()
        mine = 10.0 + 5.0 * rank  # this rank's time per step
        out[rank] = (bench.max_over_ranks(mine, dist), bench.max_over_ranks(mine, None))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    assert res[0] == (15.0, 10.0)
    assert res[1] == (15.0, 15.0)
