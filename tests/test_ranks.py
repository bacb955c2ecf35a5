"""Host logic of the multi-rank benchmark path (replicas: one tensor per rank,
no data-path collective), run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Rank r is slower on the first timing and faster on the second.
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank])
        out[rank] = (got, bench.rank_seed(rank))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        assert res[r][0] == [2.0, 10.0]
    # Each rank decomposes a different tensor.
    assert res[0][1] != res[1][1]


def test_single_process_max_is_identity():
    assert bench.max_over_ranks([3.5, 4.0]) == [3.5, 4.0]


def test_job_value_counts_every_rank():
    # Two ranks, 1e9 flops each per step, slowest rank 10 ms: 200 GFLOP/s for the job.
    assert bench.job_value(1e9, 2, 10.0) == pytest.approx(200.0)
    assert bench.job_value(1e9, 1, 10.0) == pytest.approx(100.0)
