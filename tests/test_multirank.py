"""The multi-rank (replica) bookkeeping of bench.py on two gloo ranks on the CPU: the job time
is the slowest rank's, the whole-job rate counts every replica's cells, and every rank sees
the same numbers."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]                     # rank 1 is the slower replica
    ms_max = bench.reduce_max(ms, world, torch.device("cpu"))
    out[rank] = (ms_max, bench.job_rate(world, 256**3, 4, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        ms_max, rate = out[r]
        assert ms_max == 150.0
        assert rate == pytest.approx(2 * 256**3 * 4 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max(7.0, 1, None) == 7.0
    assert bench.job_rate(1, 10, 2, 1000.0) == pytest.approx(20.0)
