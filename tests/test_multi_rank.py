"""The multi-GPU path is replicas only: ranks share no data, and the bench
reports all ranks' triangles over the slowest rank's step time.  Checked with
two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [2.0, 5.0][rank]
    units = [1000, 3000][rank]
    rate, ms_max = bench.whole_job_rate(ms, units, dist)
    dist.barrier()
    q.put((rank, rate, ms_max))
    dist.destroy_process_group()


def test_whole_job_rate_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms_max in res:
        assert ms_max == pytest.approx(5.0)
        assert rate == pytest.approx(4000 / 5e-3)


def test_whole_job_rate_single():
    import bench
    rate, ms = bench.whole_job_rate(2.0, 1000)
    assert ms == 2.0 and rate == pytest.approx(1000 / 2e-3)
