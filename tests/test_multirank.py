"""The benchmark's multi-GPU contract on CPU: N replicas (sub-traces are
independent, Sec. 3.3, so the data path has no collective), the slowest rank's
time sets the step time and the value counts every rank's instructions.  Run
as world-size-2 `gloo` process groups on 127.0.0.1."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]            # rank 1 is slower
    out = bench.aggregate(ms, steps=10, inst_per_step=1_000_000, world=world, device="cpu")
    q.put((rank, out))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms_per_step, value = res[r]
        assert ms_per_step == pytest.approx(15.0)                  # max over ranks: 150 ms / 10 steps
        assert value == pytest.approx(2 * 1_000_000 / 0.015)       # both ranks' instructions


def test_single_rank_aggregation():
    import bench
    ms_per_step, value = bench.aggregate(50.0, steps=5, inst_per_step=1000, world=1, device="cpu")
    assert ms_per_step == 10.0 and value == pytest.approx(1e5)
