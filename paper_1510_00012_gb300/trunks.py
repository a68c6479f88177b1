"""Member-parallel trunks: one B-ADMM update split over several processes.

The parallel implementation of Section 5 splits the data into trunks, one per
process; each process runs Algorithm badmm's per-member work on its own
members, and the centroid statistics are synchronised every inner iteration.
libd2 takes every cross-member sum in exact 64-bit fixed point (see
d2_set_reducer in include/d2.h), so the synchronisation is an element-wise
int64 all-reduce (sum, and max for the scales) of K m values per iteration
and K m d per support update, and the results are bitwise those of one
process holding every member -- provided the split keeps whole groups of 64
consecutive members of a cluster together (the groups whose partial sums
the library forms).

trunk_split() makes such a split; TorchReducer performs the all-reduce with
torch.distributed (NCCL for CUDA buffers), on the library's stream.  Both are
host-side plumbing: every step of the update runs in libd2's kernels.
"""
from __future__ import annotations

import torch

GROUP = 64  # members per partial-sum group of libd2 (D2_CHUNK)


def trunk_split(cluster_offsets, members, rank, world, group=GROUP):
    """This process's members: cluster c's members, in their order, cut into
    groups of `group`; group g of cluster c goes to process (g + c) mod world.
    Returns (cluster_offsets, members) int64 CPU tensors for this process."""
    co = torch.as_tensor(cluster_offsets).cpu().to(torch.int64)
    mem = torch.as_tensor(members).cpu().to(torch.int64)
    K = co.numel() - 1
    offs = [0]
    parts = []
    for c in range(K):
        a, b = int(co[c]), int(co[c + 1])
        for gi, s in enumerate(range(a, b, group)):
            if (gi + c) % world == rank:
                parts.append(mem[s:min(s + group, b)])
        offs.append(sum(p.numel() for p in parts))
    local = torch.cat(parts) if parts else torch.zeros(0, dtype=torch.int64)
    return torch.tensor(offs, dtype=torch.int64), local


class _CudaInt64View:
    """__cuda_array_interface__ of an int64 device buffer (so torch can wrap it)."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<i8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def reduce_tensor(t, op, group=None):
    """In-place element-wise sum (op 0) or max (op 1) of t across the group."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == 1 else dist.ReduceOp.SUM, group=group)
    return t


class TorchReducer:
    """Reducer for Context.set_reducer: all-reduces libd2's int64 buffers with
    torch.distributed on the stream the library works on."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, op, ptr, count, stream):
        t = torch.as_tensor(_CudaInt64View(ptr, count), device="cuda")
        s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
        with torch.cuda.stream(s):
            reduce_tensor(t, op, self.group)
        return 0
