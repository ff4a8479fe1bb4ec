"""bench.py's multi-GPU arithmetic on CPU: N independent replicas (one graph
per rank, no data exchange) report the slowest rank's time and the units of
all ranks.  Two gloo ranks stand in for two GPUs."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = bench.aggregate_replicas(dist, 100.0 + 50.0 * rank, 1024 * (rank + 1))
        out[rank] = (ms, units)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_report_slowest_time_and_all_units():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (150.0, 1024 + 2048)


def test_single_process_is_local():
    import bench
    assert bench.aggregate_replicas(None, 12.5, 7) == (12.5, 7)
