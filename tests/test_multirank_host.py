"""Host logic of the multi-GPU path on CPU ranks (gloo, world_size 2): each
rank draws its own problem from a rank-dependent seed, and the job's step
time is the slowest rank's (max over ranks), so the whole-job rate is
world x per-rank entries x T / that time.  No GPU is used."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    seed = bench.rank_seed(100, rank)
    bags, co, mem = synth.ragged_cluster_bags(seed, 3, d=4, nc=(16, 32), mk=(4, 8))
    local_ms = 10.0 + 5.0 * rank
    ms = bench.max_over_ranks(local_ms, dist)
    q.put((rank, seed, float(bags.supp.sum()), ms, bench.job_rate(1000, 100, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, sum0, ms0, v0), (r1, s1, sum1, ms1, v1) = res
    assert s0 != s1 and sum0 != sum1          # independent problems per rank
    assert ms0 == ms1 == 15.0                 # max over ranks
    assert v0 == v1 == pytest.approx(2 * 1000 * 100 / 15e-3)
