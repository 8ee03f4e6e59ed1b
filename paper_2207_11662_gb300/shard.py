"""One graph's analysis split over ranks: every rank runs the BFS from its share of the source
batches (homln_shard_partials), one element-wise sum over the ranks (an all-reduce) gives the
exact farness and reach, and every rank takes them as the graph's analysis
(homln_import_partials). The sum is exact integer arithmetic, so the result is identical to an
unsplit analysis. The reduction is torch.distributed's (NCCL for CUDA tensors, gloo for CPU).
"""
from __future__ import annotations


def reduce_partials(F, R, dist, group=None):
    """Sum the ranks' partial farness (int64) and reach (int32) in place."""
    dist.all_reduce(F, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(R, op=dist.ReduceOp.SUM, group=group)
    return F, R


def sharded_analysis(net, which: int, mask: int, dist, group=None):
    """Analyse graph `which` (layer id, -1 AND or -2 OR of `mask`) of `net` (a homln.Network)
    over the ranks of `dist`; every rank ends with the full result cached in its handle.
    Returns the reduced (farness, reach) tensors."""
    import torch

    from . import homln as H
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    F = torch.empty(net.n, dtype=torch.int64, device=net.device)
    R = torch.empty(net.n, dtype=torch.int32, device=net.device)
    H.homln_shard_partials(net.h, which, mask, rank, world, F, R)
    reduce_partials(F, R, dist, group)
    H.homln_import_partials(net.h, which, mask, F, R)
    return F, R
