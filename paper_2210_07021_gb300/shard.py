"""Sharding of independent sFMM problems over ranks (one process per GPU).

The solve has no exchange step between independent problems (sky shells or
independent skies), so N ranks each solve their own problem with no data-path
collective; the only communication is the barrier and the max-over-ranks of
the timed region that whole-job throughput needs.  Works with the gloo backend
(CPU tensors) and the nccl backend (CUDA tensors).
"""
import os


def dist_env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_config_index(base, rank):
    """Seed stream of this rank's problem: distinct per rank, rank 0 = base."""
    return base + 100 * rank


def max_over_ranks(value, device="cpu"):
    """The maximum of a float over all ranks (value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, world_size, seconds_max):
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    return units_per_rank * steps * world_size / seconds_max
