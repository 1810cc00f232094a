"""Rank bookkeeping for runs with one process per GPU (torchrun).

Independent grains shard across ranks with no data-path collective; the only
communication is a barrier around the timed region and the maximum of the
ranks' elapsed times (whole-job throughput = all ranks' work / slowest rank).
"""
import os


def env_ranks():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend="nccl"):
    """Join the process group when launched with more than one rank; returns
    the torch.distributed module or None."""
    world, _, _ = env_ranks()
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    if not dist.is_initialized():
        dist.init_process_group(backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value, device="cpu"):
    """Largest value over all ranks (the slowest rank's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank, world, slowest_seconds):
    """Whole-job rate: every rank processed units_per_rank in at most slowest_seconds."""
    return world * units_per_rank / slowest_seconds
