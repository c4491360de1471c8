"""bench.py's aggregation over replicas (one process per GPU): the job's time
is the slowest rank's, its work the sum over ranks.  Checked with two gloo
ranks on the CPU (the GPU run uses NCCL with the same calls)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, e = bench.reduce_ranks(1.0 + rank, 100.0 * (rank + 1), dist, "cpu")
        q.put((rank, t, e))
    finally:
        dist.destroy_process_group()


def test_reduce_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, e in got:
        assert t == 2.0      # the slower rank's seconds
        assert e == 300.0    # 100 + 200 edges


def test_reduce_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_ranks(1.5, 10.0, None, "cpu") == (1.5, 10.0)
