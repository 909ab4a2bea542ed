"""Several GPUs for the batched scan and for serving: independent cascades go
to GPUs by predicted work (no data-path exchange), and the only cross-rank
steps are the whole-job figures.  The assignment, the routing and the merge
are host logic, checked here on the CPU (the gather with two gloo ranks)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench_workloads as BW


def test_shard_covers_every_member_once_and_balances_the_work():
    rng = np.random.default_rng(3)
    costs = list(rng.lognormal(0.0, 1.5, 256))
    for world in (1, 2, 3, 4, 8):
        parts = BW.shard_by_work(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than the
        # largest single cost
        assert max(loads) - sum(costs) / world <= max(costs) + 1e-9
        for p in parts:
            assert p == sorted(p)


def test_shard_of_known_costs():
    # largest first: 10 -> rank 0, 7 -> 1, 6 -> 1 (7 < 10), 5 -> 0 (10 < 13),
    # 4 -> 1 (13 < 15); loads 15 and 17
    parts = BW.shard_by_work([5, 10, 4, 7, 6], 2)
    assert parts == [[0, 1], [2, 3, 4]]
    # one rank takes everything, in order
    assert BW.shard_by_work([3, 1, 2], 1) == [[0, 1, 2]]
    # more ranks than members: the surplus ranks get nothing
    assert BW.shard_by_work([1.0, 2.0], 4) == [[1], [0], [], []]
    with pytest.raises(ValueError):
        BW.shard_by_work([1.0], 0)


def test_routing_in_arrival_order():
    # loads after each request: [4,0] [4,1] [4,2] [4,5] [7,5] -> ranks 0 1 1 1 0
    assert BW.route_requests([4, 1, 1, 3, 3], 2) == [0, 1, 1, 1, 0]
    assert BW.route_requests([1, 1, 1], 1) == [0, 0, 0]
    rng = np.random.default_rng(5)
    costs = rng.lognormal(0.0, 1.0, 500)
    r = np.array(BW.route_requests(list(costs), 4))
    loads = np.array([costs[r == k].sum() for k in range(4)])
    assert loads.max() - loads.min() <= costs.max() + 1e-9


def _part(ps, wall, ttr, wait, busy=0):
    return {"particle_steps": ps, "wall_s": wall, "requests": len(ttr), "ttr": ttr, "wait": wait,
            "busy_rejections": busy}


def test_merged_serving_figures():
    a = _part(1.0e12, 10.0, [1.0, 2.0, 3.0], [0.1, 0.1, 0.2], busy=2)
    b = _part(3.0e12, 20.0, [4.0, 5.0], [0.3, 0.4], busy=1)
    m = BW.merge_served([a, b])
    assert m["particle_steps"] == 4.0e12
    assert m["wall_s"] == 20.0
    assert m["value"] == pytest.approx(2.0e11)
    assert m["requests"] == 5
    assert m["requests_per_s"] == pytest.approx(0.25)
    assert m["p50_time_to_result_s"] == pytest.approx(3.0)
    assert m["p99_time_to_result_s"] == pytest.approx(np.percentile([1, 2, 3, 4, 5], 99))
    assert m["p50_wait_for_admission_s"] == pytest.approx(0.2)
    assert m["busy_rejections"] == 3
    assert m["ranks"] == 2
    # one part: its own figures
    one = BW.merge_served([a])
    assert one["value"] == pytest.approx(1.0e11)
    assert one["p50_time_to_result_s"] == pytest.approx(2.0)


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
    import bench_workloads as W

    # every rank derives the same routing from the same trace, serves its own
    # requests, and the gathered parts merge into the whole job's figures
    costs = [4.0, 1.0, 1.0, 3.0, 3.0, 2.0]
    route = W.route_requests(costs, world)
    mine = [i for i, k in enumerate(route) if k == rank]
    part = _part(sum(costs[i] for i in mine) * 1e10, 5.0 + rank, [float(i) for i in mine], [0.0] * len(mine))
    merged = W.merge_served(W._gather(part, world))
    out[rank] = (route, merged["particle_steps"], merged["wall_s"], merged["requests"])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_serving_gather():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0]  # the same routing on both ranks
    for r in (r0, r1):
        assert r[1] == pytest.approx(14.0e10)
        assert r[2] == 6.0
        assert r[3] == 6
