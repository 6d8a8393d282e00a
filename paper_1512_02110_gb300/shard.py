"""Photon-id sharding across processes (Sec. 1: photon packets are independent).

A render of N photons splits into ranks that trace disjoint id ranges with the same
normaliser N (mst_params.photon_offset / n_photons / n_photons_total). The per-rank L and
replay gradients then sum exactly to the single-process result, so a multi-GPU job needs one
sum-reduction of L (C x nvox FP64) after transport and one of the gradient (nvox) after the
replay; the benchmark instead gives every rank its own photons (weak scaling, no collective).
"""
from __future__ import annotations


def shard(n_total: int, rank: int, world: int):
    """(photon_offset, n_photons) of `rank` when n_total photons are split over `world` ranks:
    contiguous ranges, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, rem = divmod(int(n_total), int(world))
    count = base + (1 if rank < rem else 0)
    offset = rank * base + min(rank, rem)
    return offset, count


def allreduce_sum_(tensor, group=None):
    """In-place sum over ranks (torch.distributed), a no-op without a process group."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor
