"""The multi-rank path of the benchmark on CPU: two gloo ranks each build an
independent problem (distinct seeds, no data exchange) and agree on the
slowest rank's time, from which the whole-job rate is formed."""
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
