"""The benchmark's N > 1 path on CPU: two `gloo` ranks reduce their timings to the
slowest rank and their work to the sum, and draw disjoint problem sets (weak
scaling: independent problems, no data-path collective)."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    device_s, wall_s, units = bench.reduce_over_ranks(dist, torch, 0.5 + rank, 2.0 - rank, 100 * (rank + 1), "cpu")
    out[rank] = (device_s, wall_s, units, bench.rank_problem_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_sum_work():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        device_s, wall_s, units, seed = res[rank]
        assert device_s == 1.5 and wall_s == 2.0 and units == 300.0
    seeds = [res[r][3] for r in range(world)]
    assert len(set(seeds)) == world and all(b - a >= 10000 for a, b in zip(seeds, seeds[1:]))


def test_single_process_passes_values_through():
    import bench
    assert bench.reduce_over_ranks(None, torch, 0.25, 1.0, 42, "cpu") == (0.25, 1.0, 42)


def _rank_plan_main(rank, world, port, count, out):
    """One rank of the weak-scaling layout: plan this rank's own problems (the
    oracle stands in for the device planner on CPU), then reduce the time to the
    slowest rank and the work to the sum -- the only collective."""
    import time

    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    probs = bench.shelf_problems(O.accept, count=count, seed0=bench.rank_problem_seed(rank))
    t = time.perf_counter()
    rs = O.plan_batch(probs, threads=1, seed=1, problem_ids=[rank * count + k for k in range(count)], range=1.0,
                      resolution=float(np.float32(1 / 32)), goal_bias=float(np.float32(0.05)))
    wall = time.perf_counter() - t
    units = sum(r["states_checked"] for r in rs)
    device_s, wall_s, total = bench.reduce_over_ranks(dist, torch, wall, wall, units, "cpu")
    out[rank] = dict(seeds=[p.seed for p in probs], costs=[r["cost"] for r in rs], status=[r["status"] for r in rs],
                     units=units, wall=wall, total=total, device_s=device_s)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_plan_disjoint_shards():
    """Two ranks plan disjoint problem sets; the reduced work is the sum of what
    each rank planned, the reduced time the slower rank's; each rank's plans equal
    a single-process run of the same shard."""
    import numpy as np

    import bench
    from oracle import oracle as O
    world, count = 2, 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_plan_main, args=(world, port, count, out), nprocs=world, join=True)
        res = dict(out)
    assert not set(res[0]["seeds"]) & set(res[1]["seeds"])
    total = res[0]["units"] + res[1]["units"]
    for r in range(world):
        assert res[r]["total"] == total
        assert res[r]["device_s"] == max(res[0]["wall"], res[1]["wall"])
    for r in range(world):
        probs = bench.shelf_problems(O.accept, count=count, seed0=bench.rank_problem_seed(r))
        alone = O.plan_batch(probs, threads=1, seed=1, problem_ids=[r * count + k for k in range(count)], range=1.0,
                             resolution=float(np.float32(1 / 32)), goal_bias=float(np.float32(0.05)))
        assert [a["status"] for a in alone] == res[r]["status"]
        assert [a["cost"] for a in alone] == res[r]["costs"]
