"""The multi-GPU path of bench.py is replicas (one independent elimination
per rank, no data-path collective): the whole-job rate is world x work over
the slowest rank's time.  Checked here with two CPU ranks over gloo."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [100.0, 250.0][rank]
    rate, max_ms = bench.replica_rate(local_ms, 1.0e12, world, torch.device("cpu"))
    out[rank] = (rate, max_ms)
    dist.destroy_process_group()


def test_replica_rate_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        rate, max_ms = res[r]
        assert max_ms == 250.0
        assert rate == pytest.approx(2 * 1.0e12 / 0.250)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    rate, max_ms = bench.replica_rate(500.0, 2.0e12, 1, None)
    assert max_ms == 500.0 and rate == pytest.approx(4.0e12)
