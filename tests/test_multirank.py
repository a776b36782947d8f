"""The N > 1 form of the benchmark on CPU ranks (gloo, world size 2).

The path shards by replicas: every rank runs its own copy of the workload and
there is no collective on the data path.  The job's step time is the maximum
over ranks and its throughput counts the queries of all ranks.
"""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ms_by_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.job_ms(ms_by_rank[rank], dist)
    out[rank] = (ms, bench.job_value(world, 10_000, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_time_is_the_max_and_value_counts_all_ranks():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ms_by_rank = [800.0, 1000.0]
    mp.spawn(_worker, args=(2, _free_port(), ms_by_rank, out), nprocs=2, join=True)
    for r in range(2):
        ms, value = out[r]
        assert ms == 1000.0
        assert value == pytest.approx(2 * 10_000 / 1.0)


def test_single_rank_passthrough():
    import bench
    assert bench.job_ms(123.0, None) == 123.0
    assert bench.job_value(1, 500, 250.0) == pytest.approx(2000.0)
