"""The multi-GPU path of bench.py on CPU: ranks as gloo processes (world size
2) run independent replicas; the job's time is the slowest rank's and its
rate counts every rank's pixels.  No collective touches the data path."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    local_ms = 10.0 + 5.0 * rank            # rank 1 is the slower replica
    total = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.job_rate(4096 * 4096, world, 100, total)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, total, rate))


def test_two_rank_replicas_max_time_and_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total, rate in res:
        assert total == 15.0                  # max over ranks on every rank
        assert rate == pytest.approx(4096 * 4096 * 2 * 100 / 0.015 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(1000, 1, 10, 1.0) == pytest.approx(10.0)
