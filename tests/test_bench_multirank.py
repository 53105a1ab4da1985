"""The N > 1 path of bench.py (independent replicas, one per rank) on CPU with gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    value, ms_max, ws = bench.aggregate_replicas(local_ms, 1.0e9)
    out[rank] = (value, ms_max, ws)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_takes_max_time_and_sums_units():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, ms_max, ws = res[rank]
        assert ws == world
        assert ms_max == pytest.approx(200.0)
        assert value == pytest.approx(2.0e9 / 0.2)


def test_single_process_aggregation():
    import bench
    value, ms_max, ws = bench.aggregate_replicas(50.0, 1.0e6)
    assert ws == 1 and ms_max == 50.0 and value == pytest.approx(2.0e7)
