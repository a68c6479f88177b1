"""Host logic of the member-parallel trunks on two gloo ranks (CPU): the split
keeps whole groups of 64 consecutive members of a cluster, every member lands
on exactly one rank in its cluster, and the reducer's all-reduce sums and
takes maxima of int64 buffers element-wise (the reduction libd2 asks for)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1510_00012_gb300.trunks import GROUP, reduce_tensor, trunk_split


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _clustering():
    g = torch.Generator().manual_seed(3)
    sizes = torch.tensor([1, 64, 65, 200, 7, 128, 300, 0, 63])
    co = torch.zeros(sizes.numel() + 1, dtype=torch.int64)
    co[1:] = torch.cumsum(sizes, 0)
    members = torch.randperm(int(co[-1]), generator=g)
    return co, members


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        co, members = _clustering()
        lco, lmem = trunk_split(co, members, rank, world)
        pieces = [lmem[int(lco[c]):int(lco[c + 1])].tolist() for c in range(co.numel() - 1)]
        # element-wise sum and max across ranks
        a = torch.tensor([rank + 1, -5 * rank, 1 << 40, rank], dtype=torch.int64)
        s = reduce_tensor(a.clone(), 0)
        mx = reduce_tensor(a.clone(), 1)
        out.put((rank, pieces, s.tolist(), mx.tolist()))
    finally:
        dist.destroy_process_group()


def test_trunk_split_and_reduce_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict()
    for _ in range(world):
        r, pieces, s, mx = q.get(timeout=120)
        res[r] = (pieces, s, mx)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    co, members = _clustering()
    for c in range(co.numel() - 1):
        ids = members[int(co[c]):int(co[c + 1])].tolist()
        groups = [ids[s:s + GROUP] for s in range(0, len(ids), GROUP)]
        for r in range(world):
            mine = [g for gi, g in enumerate(groups) if (gi + c) % world == r]
            assert res[r][0][c] == sum(mine, [])           # whole groups, in order
        assert sorted(res[0][0][c] + res[1][0][c]) == sorted(ids)
    assert res[0][1] == res[1][1] == [3, -5, 2 << 40, 1]
    assert res[0][2] == res[1][2] == [2, 0, 1 << 40, 1]
