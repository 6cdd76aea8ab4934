"""Photon-range sharding across ranks (one process per GPU).

Photons are independent and their random streams are keyed by photon id, so a
run of `per_rank * world` photons splits into disjoint id ranges, one per rank,
with no data-path communication. Each rank normalises its fields with the
photon count of the whole run (photons_total), so summing the ranks' fields
(reduce_fields: one sum all-reduce per field, NCCL between GPUs) reproduces
the single-process run up to the order of FP64 additions.
"""
from __future__ import annotations


def photon_range(rank: int, world: int, per_rank: int) -> tuple[int, int, int]:
    """(begin, count, total) of this rank's photon ids for weak scaling."""
    if world <= 0 or not 0 <= rank < world or per_rank < 0:
        raise ValueError("need 0 <= rank < world and per_rank >= 0")
    return rank * per_rank, per_rank, per_rank * world


def split_range(rank: int, world: int, total: int) -> tuple[int, int, int]:
    """(begin, count, total) of this rank's share of a fixed total (strong scaling)."""
    if world <= 0 or not 0 <= rank < world or total < 0:
        raise ValueError("need 0 <= rank < world and total >= 0")
    base, rem = divmod(total, world)
    begin = rank * base + min(rank, rem)
    return begin, base + (1 if rank < rem else 0), total


def sum_tallies(arrays, group=None):
    """In-place sum of a list of torch tensors over the process group."""
    import torch.distributed as dist
    for a in arrays:
        dist.all_reduce(a, op=dist.ReduceOp.SUM, group=group)
    return arrays


def reduce_fields(fields, group=None):
    """Sum the output fields of all ranks in place (dict or list of tensors).

    The fields must be normalised with the whole run's photon count, as
    rt_trace_range does with photons_total; absorption, fluxes and heating
    rates are all linear in the tallies, so their sums are the fields of the
    combined run. Returns the same container.
    """
    import torch.distributed as dist
    tensors = list(fields.values()) if isinstance(fields, dict) else list(fields)
    for a in tensors:
        dist.all_reduce(a, op=dist.ReduceOp.SUM, group=group)
    return fields
