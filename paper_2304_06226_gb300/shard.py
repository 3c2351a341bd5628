"""Sharding of histories over GPUs and the reduction of their tallies.

Histories are independent and their random numbers are keyed by history id
(Philox counter = (event, sub-stream, history id, instance)), so a run over
disjoint id ranges on several GPUs gives, summed, exactly the tallies of one
run over all ids.  Each rank transports a contiguous id range; the partial
accumulators -- FP64 sum w, sum w^2 per bin, the score-function tallies J, J2
and the history count per instance -- are combined by one sum all-reduce in
FP64 (torch.distributed: NCCL on GPUs, gloo on CPUs).  Nothing else crosses
ranks.  Argument handling only: the transport runs in the CUDA kernels."""
from __future__ import annotations

import torch


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """(first id, count) of rank's contiguous share of n_total history ids;
    the shares differ by at most one history and cover [0, n_total)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    lo = n_total * rank // world
    hi = n_total * (rank + 1) // world
    return lo, hi - lo


def step_stream(step: int, rank: int, world: int, n_per_rank: int, seed: int) -> tuple[int, int]:
    """(Philox key, first history id) of `rank` at `step` when every rank runs
    n_per_rank histories per step (weak scaling), so that no history is ever
    repeated across steps or ranks: each step takes its own key (seed + step),
    and within a step the ranks take consecutive id ranges while all of them
    fit below 2^32 (history ids are 32-bit counter words); beyond that each
    rank takes its own key as well."""
    if world * n_per_rank <= 2 ** 32:
        return seed + step, rank * n_per_rank
    return seed + step * world + rank, 0


def reduce_sums(parts: dict, group=None) -> dict:
    """Sum-all-reduce of partial accumulators over the ranks of `group`.

    parts: name -> FP64 tensor (sum, sumsq, J, J2 as [n_inst, bins] or
    [n_par, n_inst, bins], n as [n_inst]); all ranks pass the same names and
    shapes.  The tensors are packed into one buffer so that the reduction is a
    single collective, reduced in FP64 and unpacked in place; returns parts."""
    import torch.distributed as dist
    names = sorted(parts)
    for k in names:
        if parts[k].dtype != torch.float64:
            raise TypeError(f"{k}: the tallies reduce in FP64, got {parts[k].dtype}")
    flat = torch.cat([parts[k].reshape(-1) for k in names])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    o = 0
    for k in names:
        n = parts[k].numel()
        parts[k].copy_(flat[o:o + n].view_as(parts[k]))
        o += n
    return parts
