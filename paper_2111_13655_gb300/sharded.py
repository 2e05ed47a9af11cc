"""Term-sharded H_S x over the ranks of a torch.distributed group (one GPU each).

Every rank holds a context of the same problem and the same input vectors.
Rank r adds the terms at processing positions p = r (mod world) into int64
fixed-point accumulators (sg_apply_H_part); one all-reduce (sum) of the
accumulators -- the paper's MPI sum of partial results (Alg. 2) -- and
sg_apply_H_finish give every rank y, bitwise the single-GPU sg_apply_H
whatever the number of ranks (integer sums are associative).  Integer sums
that overflow wrap modulo 2^64 on every backend used here; the final value
fits, so wrapped partial sums are harmless.
"""
from __future__ import annotations

import paper_2111_13655_gb300 as sg


def reduce_accumulators(acc, group=None):
    """Sum of the ranks' int64 accumulators, in place (one collective)."""
    import torch.distributed as dist
    dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    return acc


def apply_H_sharded(ctx, x, y, nvec: int, acc=None, group=None, stream=None):
    """y = H_S x with this rank's share of the terms; acc (int64 CUDA tensor of
    sg.acc_words(ctx, nvec) zeros) may be passed in to reuse it."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    if acc is None:
        acc = torch.zeros(sg.acc_words(ctx, nvec), dtype=torch.int64, device=x.device)
    sg.sg_apply_H_part(ctx, x, acc, nvec, rank, world, stream)
    if world > 1:
        reduce_accumulators(acc, group)
    sg.sg_apply_H_finish(ctx, x, acc, y, nvec, stream)
    return acc
