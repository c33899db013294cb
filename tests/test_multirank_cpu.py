"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): every
rank runs its own replica, the job's time is the slowest rank's, and the
job's rate sums the ranks' units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, lr = bench.dist_env()
    assert (w, r, lr) == (world, rank, rank)
    bench.barrier(world)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slowest
    rate, ms_job = bench.job_rate(1000, ms, world)
    out[rank] = (rate, ms_job)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        rate, ms_job = out[rank]
        assert ms_job == 15.0
        assert abs(rate - 2000 / 15e-3) < 1e-6
