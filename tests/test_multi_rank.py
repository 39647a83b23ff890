"""The N > 1 path of the benchmark on CPU: two gloo ranks, each with its own problem seed,
combine their timings into the whole-job rate (point-steps summed over ranks, time of the
slowest rank).  No GPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2507_23613_gb300 import multi


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 100.0 + 50.0 * rank          # ms: rank 1 is the slowest
        pts = 1e9 * (rank + 1)
        value, t_max, total = multi.weak_scaling_rate(elapsed, pts, dist, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, multi.problem_seed(2000, rank))
        out[rank] = (value, t_max, total, tuple(seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_timings():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, t_max, total, seeds = res[rank]
        assert t_max == 150.0 and total == 3e9
        assert abs(value - 3e9 / 0.150 / 1e9) < 1e-9
        assert len(set(seeds)) == world
    # one process: the rate of its own numbers
    assert multi.weak_scaling_rate(200.0, 4e9)[0] == pytest.approx(20.0)
