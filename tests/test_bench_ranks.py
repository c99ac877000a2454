"""The bench's replica aggregation (the N > 1 path, replicas only) on two
gloo ranks on the CPU: the job's time is the slowest rank's, its updates the
sum over the ranks, and the barrier around the timed steps releases both."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        # rank r: 1.5 + r seconds over 1000 (r + 1) point updates
        cells, t = bench.aggregate_ranks(1.5 + rank, 1000 * (rank + 1), "cpu")
        dist.barrier()
        out[rank] = (cells, t)
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
    for r in range(2):
        cells, t = out[r]
        assert cells == 3000.0 and t == 2.5


def test_single_process_is_local():
    sys.path.insert(0, ROOT)
    import bench

    assert not dist.is_initialized()
    assert bench.aggregate_ranks(0.75, 1234, "cpu") == (1234.0, 0.75)
