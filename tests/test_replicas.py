"""Multi-GPU runs are independent replicas (the method has no exchange
between separate runs): bench.py's rank aggregation -- the slowest rank's
time, all ranks' cell updates -- checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [10.0 + 5.0 * rank, 2.0 - rank]  # per-rank (timed ms, e2e s)
    out[rank] = bench.max_over_ranks(mine, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks_and_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == [15.0, 2.0]
    import sys
    sys.path.insert(0, ROOT)
    import bench
    # 2 replicas of 1000 cells, 10 steps each, slowest rank 15 ms
    assert abs(bench.job_mlups(1000, 10, 2, 15.0) - 2 * 1000 * 10 / 0.015 / 1e6) < 1e-12

