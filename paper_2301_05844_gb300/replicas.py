"""Multi-GPU layout of the workload: independent replicas, one process per GPU.

Every message of a sweep is computed from the previous sweep's messages only (Eq. 1),
so whole solves are independent units: N ranks run N solves (the same lattice, or
different requests of a served mix) with no exchange on the data path.  The only
collectives are the barrier around the timed region and the maximum of the per-rank
device time, from which the whole-job throughput is taken.
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, local_rank, world_size) from the torchrun environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard(items, rank, world):
    """Round-robin share of a list of independent units (e.g. the requests of a served
    mix) for one rank; the shares of all ranks partition the list."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(items[rank::world])


def max_over_ranks(seconds, device=None):
    """Maximum of a per-rank duration over all ranks (the job takes as long as its
    slowest rank).  Without an initialised process group it returns its argument."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, slowest_seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    if slowest_seconds <= 0:
        raise ValueError("duration must be positive")
    return units_per_rank * world / slowest_seconds
