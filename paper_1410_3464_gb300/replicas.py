"""Replica bookkeeping for runs on several GPUs of one node.

Simulations are independent of one another, so N GPUs run N replicas (or N
disjoint shares of a request list) with no exchange on the data path.  Only the
timing crosses ranks: a barrier before and after the timed region and the
maximum of the per-rank times, from which the whole-job rate is computed.
Rank, world size and rendezvous come from the environment that
torch.distributed.run sets (RANK, LOCAL_RANK, WORLD_SIZE, MASTER_ADDR,
MASTER_PORT).
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world_size):
    """Join the gloo process group when there is more than one rank."""
    if world_size > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("gloo", init_method="env://")


def barrier(world_size):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world_size):
    """Largest value over all ranks (the slowest rank's time)."""
    if world_size <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world_size, max_seconds):
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * world_size / max_seconds


def share(items, rank, world_size):
    """The items rank `rank` takes of a list split round-robin over the ranks
    (independent requests or batch members; every item goes to exactly one
    rank)."""
    return items[rank::world_size]


def finish(world_size):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
