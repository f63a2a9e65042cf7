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
