"""The multi-GPU form of the benchmark runs independent replicas; its only
cross-rank step is the whole-job aggregation (slowest rank's time, all ranks'
particle-steps).  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [120.0, 150.0][rank]
    ps = [1.0e12, 1.2e12][rank]
    t, p = bench.aggregate_over_ranks(ms, ps, "cpu")
    out[rank] = (t, p)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in (0, 1):
        t, p = out[r]
        assert t == 150.0
        assert p == pytest.approx(2.2e12)


def test_single_rank_aggregation_is_identity():
    import bench

    assert bench.aggregate_over_ranks(5.0, 7.0, "cpu") == (5.0, 7.0)
