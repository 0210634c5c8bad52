"""The N > 1 benchmark path on CPU: world-size-2 gloo ranks run the benchmark's rank
aggregation (max over ranks of the timed region, whole-job replica throughput), and the
reference arm does no work on ranks other than 0. No GPU, no NCCL."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 1000.0 + 250.0 * rank  # rank 1 is the slow one
    t_max = bench.max_over_ranks(local_ms, world, "cpu")
    value = bench.replica_throughput(world, 4, t_max)
    dist.barrier()

    class A:
        steps, warmup, ref_matvecs = 1, 0, 1
    ref = bench.run_reference(A(), rank, world) if rank != 0 else "rank0"
    out[rank] = (t_max, value, ref is None)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 1250.0  # both ranks see the slowest rank's time
    assert out[0][1] == out[1][1] == pytest.approx(2 * 4 / 1.25)  # 2 replicas x 4 solves in 1.25 s
    assert out[1][2]  # the reference arm returns without work on rank 1


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_throughput(1, 3, 1500.0) == pytest.approx(2.0)
