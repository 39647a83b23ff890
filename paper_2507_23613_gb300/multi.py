"""Host logic of multi-GPU runs: one process per GPU, each solving its own independent
MFWH problem (no data-path collective), whole-job rate from the slowest rank.

The map Pi is one time-stepping recurrence per problem; independent problems shard across
GPUs with nothing to exchange, so N GPUs run N problems (weak scaling).  The only
collectives are the two reductions of the timing below.
"""


def problem_seed(base, rank):
    """Seed of the problem a rank solves: distinct per rank."""
    return int(base) + int(rank)


def weak_scaling_rate(elapsed_ms, point_steps, dist=None, device="cpu"):
    """(Gpts/s, max elapsed ms, total point-steps) over all ranks: point-steps summed over
    ranks divided by the largest elapsed time of any rank.  dist: torch.distributed when
    initialised (any backend), else None for a single process."""
    if dist is None or not dist.is_initialized():
        return point_steps / (elapsed_ms * 1e-3) / 1e9, float(elapsed_ms), float(point_steps)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(point_steps)], dtype=torch.float64, device=device)
    dist.all_reduce(p)
    t_max, total = float(t.item()), float(p.item())
    return total / (t_max * 1e-3) / 1e9, t_max, total
