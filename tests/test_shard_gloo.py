"""The multi-rank paths on CPU: two gloo ranks each build an independent
problem (distinct seeds, no data exchange) and agree on the slowest rank's
time, from which the whole-job rate is formed; a shell set of uneven sizes is
split by the longest-first rule, each rank computing the same assignment on its
own, every shell solved exactly once and the loads balanced."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2210_07021_gb300 import shard, workloads
    ws, r, _ = shard.dist_env()
    d = workloads.clustered_pair(n=2000, n_clumps=5, config_index=shard.rank_config_index(3, r))
    fake_seconds = 1.0 + r                       # the slower rank decides the job time
    tmax = shard.max_over_ranks(fake_seconds)
    rate = shard.whole_job_rate(d["tgt"].shape[0], 3, ws, tmax)
    out[r] = (float(d["src"][0, 0]), tmax, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] != out[1][0]                 # independent problems
    assert out[0][1] == out[1][1] == 2.0          # max over ranks
    assert out[0][2] == out[1][2] == 2000 * 3 * 2 / 2.0


def test_single_process_fallbacks():
    from paper_2210_07021_gb300 import shard
    assert shard.max_over_ranks(3.5) == 3.5
    assert shard.rank_config_index(3, 0) == 3 and shard.rank_config_index(3, 1) != 3


def _shell_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2210_07021_gb300 import shard, workloads
    ws, r, _ = shard.dist_env()
    sizes = workloads.shell_sizes()                          # the 64 shells of the batched workload
    M = 786_432
    costs = [shard.shell_cost(n, M) for n in sizes]
    mine = shard.assign_shells(costs, ws)[r]
    # every rank's own list, gathered: they must partition the shells
    lists = [None] * ws
    dist.all_gather_object(lists, mine)
    load = sum(costs[i] for i in mine)
    done = shard.sum_over_ranks(len(mine) * M)                # targets solved by the whole job
    out[r] = (lists, load, shard.max_over_ranks(load), done)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shells_split_exactly_once_and_balanced(world):
    from paper_2210_07021_gb300 import shard, workloads
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_shell_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    sizes = workloads.shell_sizes()
    costs = [shard.shell_cost(n, 786_432) for n in sizes]
    lists = out[0][0]
    assert all(out[r][0] == lists for r in range(world))      # the ranks agree without an exchange
    flat = sorted(i for x in lists for i in x)
    assert flat == list(range(len(sizes)))                    # every shell exactly once
    loads = [out[r][1] for r in range(world)]
    lower = max(sum(costs) / world, max(costs))               # no assignment beats this
    assert max(loads) <= (4 / 3 - 1 / (3 * world)) * lower + 1e-6 * sum(costs)
    assert out[0][2] == max(loads)
    assert out[0][3] == len(sizes) * 786_432


def test_longest_first_assignment_cases():
    from paper_2210_07021_gb300 import shard
    assert shard.assign_shells([5, 4, 3, 3, 2, 1], 1) == [[0, 1, 2, 3, 4, 5]]
    a = shard.assign_shells([7, 7, 6, 5, 5, 4], 3)
    assert sorted(i for x in a for i in x) == list(range(6))
    assert max(sum([7, 7, 6, 5, 5, 4][i] for i in x) for x in a) == 12   # optimal here: 12, 12, 10 -> 7+5, 7+5, 6+4
    assert shard.assign_shells([1.0], 4) == [[0], [], [], []]  # more ranks than shells: idle ranks
    with pytest.raises(ValueError):
        shard.assign_shells([1.0], 0)
