"""The multi-rank path of bench.py (independent replicas, no collective on
the method's path): whole-job throughput = world x units / slowest rank's
time.  Run as two gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        # rank r took (1 + r) seconds for its 50 units, and 3 + r seconds for a second measurement
        vals, times = bench.replica_aggregate([1.0 + rank, 3.0 + rank], 50, dist, torch.device("cpu"))
        out[rank] = (vals, times)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        vals, times = res[rank]
        assert times == [2.0, 4.0]  # max over ranks
        assert vals == [2 * 50 / 2.0, 2 * 50 / 4.0]


def test_single_process_needs_no_collective():
    import bench

    vals, times = bench.replica_aggregate(0.5, 10)
    assert times == [0.5] and vals == [20.0]
