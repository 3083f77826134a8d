"""Sharding of feasibility checks over ranks (one process per GPU).

The checks of a batch are independent (Sec. 3.1: each bound is a function of
one reduced instance), so a batch shards over ranks with no data-path
exchange: rank i evaluates its own checks and keeps its own outputs.  The
work of a check is its item-parameter evaluations, r * P(c) (r reduced
items, P(c) the parameters of the six DFFs), and the shards are balanced by
that estimate.

One instance too large for one GPU shards instead over its flattened
parameter index g (DFFs in paper order, lambda ascending): every rank takes a
contiguous range of g, forms the packed key (bound << 32 | (2^32 - 1 - g)) of
its best parameter, and the bound and its first argmax are the maximum key
over ranks -- one 8-byte MAX all-reduce, the only collective of the path.

Host logic only; the evaluation itself is the C ABI's (bp_lb_eval_batch and
the other batched calls for whole checks, bp_lb_eval_range for a range of one
check's parameters).
"""
from __future__ import annotations

import numpy as np


def param_counts(c: int):
    """Parameters of each DFF at capacity c (the library's ranges, Sec. 3.1)."""
    from . import binding
    return [binding.bp_lb_param_count(d, int(c))[0] for d in range(6)]


def check_work(r, c) -> np.ndarray:
    """Estimated work of each check: r * P(c) item-parameter evaluations."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    p = np.array([sum(param_counts(int(x))) for x in c], dtype=np.int64)
    return r * p


def partition_by_work(work, world: int):
    """Splits checks 0..B-1 into `world` shards of nearly equal total work:
    longest-processing-time first, each check to the currently lightest rank.
    Returns one sorted index array per rank (every check in exactly one)."""
    work = np.asarray(work, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-work, kind="stable")
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(len(work), dtype=np.int64)
    for i in order:
        k = int(np.argmin(load))
        owner[i] = k
        load[k] += work[i]
    return [np.nonzero(owner == k)[0] for k in range(world)]


def param_ranges(total: int, world: int):
    """Contiguous ranges [g0, g1) of the flattened parameter index, one per rank."""
    bounds = [total * k // world for k in range(world + 1)]
    return [(bounds[k], bounds[k + 1]) for k in range(world)]


def make_key(bound: int, g: int) -> int:
    return (int(bound) << 32) | (0xFFFFFFFF - int(g))


def split_key(key: int):
    """(bound, g) of a packed key."""
    return int(key) >> 32, 0xFFFFFFFF - (int(key) & 0xFFFFFFFF)


def rank_key(h, sizes, c: int, rank: int, world: int, stream=None) -> int:
    """This rank's packed key for one instance: its contiguous range of the
    flattened parameter index, evaluated on this rank's GPU through the C ABI
    (bp_lb_eval_range).  `sizes` is the reduced instance as an int32 CUDA
    tensor.  The MAX over ranks (allreduce_max_key) is the full bound and its
    first argmax."""
    import torch
    from . import binding
    g0, g1 = param_ranges(sum(param_counts(c)), world)[rank]
    out = torch.empty(1, dtype=torch.int64, device=sizes.device)
    binding.bp_lb_eval_range(h, sizes, c, g0, g1, out, stream)
    return int(out.item())


def allreduce_max_key(key: int, group=None) -> int:
    """The maximum packed key over ranks: one 8-byte MAX all-reduce."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([int(key)], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return int(t.item())


def max_over_ranks(x: float, group=None) -> float:
    """Slowest rank's time (the step time of a sharded batch)."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
