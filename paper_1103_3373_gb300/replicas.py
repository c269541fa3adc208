"""Replica coordination for the multi-GPU form.

The patch groups of a step are independent (Sec. 3.1: one thread block per
group), so the path shards across GPUs with no exchange on the data path:
each rank (one process per GPU) advances its own boxes or its own share of
a group list, and only the timing is combined.  The paper's own multi-GPU
runs add a halo exchange of a domain decomposition (Sec. 4.3); for
independent replicas there is none.

    rank_info()            (rank, world, local_rank) from the launcher's env
    shard(n, rank, world)  contiguous share [start, stop) of n items
    job_rate(...)          barrier, max of the ranks' times, whole-job rate
"""
import os


def rank_info(env=None):
    env = os.environ if env is None else env
    return int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0"))


def shard(n, rank, world):
    """Contiguous share of n items for `rank` of `world`; shares differ by at
    most one item and cover [0, n) in rank order."""
    if world <= 0 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    per, extra = divmod(n, world)
    start = rank * per + min(rank, extra)
    return start, start + per + (1 if rank < extra else 0)


def job_rate(local_ms, local_units, dist=None, device="cpu"):
    """Whole-job rate of a timed region: every rank passes its own elapsed
    milliseconds and the units it processed; after a barrier the maximum time
    over ranks and the sum of units give units per second for the job.
    Returns (rate, max_ms, total_units).  Without a process group the local
    figures are returned."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_units / (local_ms / 1e3), float(local_ms), float(local_units)
    import torch
    dist.barrier()
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    max_ms, units = float(t.item()), float(u.item())
    return units / (max_ms / 1e3), max_ms, units
