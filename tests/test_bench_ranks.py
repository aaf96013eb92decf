"""The multi-rank bookkeeping of bench.py (replicas: one independent
workload per rank) on CPU with gloo, world size 2: timings are reduced by
maximum and the job value counts every rank's steps."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = [100.0 + 10 * rank, 5.0 - rank, 7.0 * (rank + 1)]
    agg = bench.max_over_ranks(mine, ws)
    q.put((rank, agg, bench.job_value(10, ws, agg[0])))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, agg, val in out:
        assert agg == [110.0, 5.0, 14.0]
        assert val == pytest.approx(2 * 10 / 0.110)


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.job_value(4, 1, 2000.0) == pytest.approx(2.0)
