"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path
collective) agree on the slowest rank's time, and the whole-job rate counts
the units of every rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_env() == (rank, world, rank)
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    mx = bench.reduce_max(ms)
    out[rank] = mx
    out[2 + rank] = bench.whole_job_rate(5 * 10, world, mx)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_max_time_and_whole_job_rate():
    world, port = 2, _free_port()
    out = torch.zeros(4, dtype=torch.float64).share_memory_()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0].item() == out[1].item() == 150.0
    # 2 ranks x 50 CGLS iterations in 150 ms
    assert out[2].item() == pytest.approx(2 * 50 / 0.150)
    assert out[3].item() == out[2].item()


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(12.5) == 12.5
    assert bench.whole_job_rate(50, 1, 1000.0) == 50.0
