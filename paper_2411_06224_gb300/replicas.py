"""Multi-GPU as independent replicas.

A single system's solve does not shard without a halo exchange every SpMV,
so N GPUs run N independent workloads: rank r solves its own seeded systems
(or its share of a batch) and no collective touches the data path.  The only
collectives are for timing: a barrier around the timed region and the
maximum of the per-rank elapsed times.  Throughput counts the units all
ranks processed divided by that maximum (weak scaling).
"""

import torch
import torch.distributed as dist


def shard(items, rank, world):
    """Round-robin share of a list of independent systems for this rank."""
    return [it for i, it in enumerate(items) if i % world == rank]


def max_over_ranks(seconds, device=None):
    """Largest elapsed time over all ranks (identity without a process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank, seconds, device=None):
    """(whole-job units per second, max elapsed) for equal per-rank work."""
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    tmax = max_over_ranks(seconds, device)
    return units_per_rank * world / tmax, tmax
