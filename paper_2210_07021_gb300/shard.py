"""Sharding of independent sFMM problems over ranks (one process per GPU).

The solve has no exchange step between independent problems (the sky shells
of the multi-plane setting, Sec. 2.1, or independent skies), so N ranks each
solve their own problems with no data-path collective; the only
communication is the barrier and the max-over-ranks of the timed region that
whole-job throughput needs.  A set of shells of very uneven sizes is split by
the longest-first greedy rule (each shell, largest cost first, goes to the
rank with the least cost so far), which every rank computes on its own from
the shell sizes, so the ranks agree without exchanging the assignment.  Works
with the gloo backend (CPU tensors) and the nccl backend (CUDA tensors).
"""
import heapq
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


def shell_cost(n_sources, n_targets):
    """Relative cost of one shell's solve: the tree, expansions and near field
    grow about linearly in the sources and the evaluation in the targets."""
    return float(n_sources) + float(n_targets)


def assign_shells(costs, world_size):
    """Longest-first greedy assignment of shells to ranks: a list (one per
    rank) of shell indices.  Deterministic: cost ties go to the lower shell
    index, load ties to the lower rank.  Its largest load is at most
    4/3 - 1/(3 world_size) times the optimal one (Graham 1969)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world_size)]
    out = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in out]


def sum_over_ranks(value, device="cpu"):
    """The sum of a float over all ranks (value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
