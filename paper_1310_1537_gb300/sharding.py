"""Row sharding of one evaluation across ranks (one GPU per rank).

The likelihood sums over disjoint row blocks add up to the whole-data sums,
so a dataset too large for one device, or a chain spread over several, can
be evaluated shard by shard and combined by one sum all-reduce of K x (P+1)
values: f (FP64) and g. The prior must be counted once: rank 0's handle keeps
it, every other rank's handle is created with GLM_FLAG_NO_PRIOR. This is the
one-combine-per-worker reduction of the paper's gradient routine (§4.2.2)
with ranks in place of threads; the evaluation itself runs in the library on
each rank.
"""
from __future__ import annotations

from . import GLM_FLAG_NO_PRIOR


def shard_rows(n_rows: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced row block [r0, r1) of `rank` among `world` ranks."""
    if world < 1 or not 0 <= rank < world or n_rows < 0:
        raise ValueError("bad shard request")
    return (n_rows * rank) // world, (n_rows * (rank + 1)) // world


def shard_flags(rank: int, flags: int = 0) -> int:
    """Handle flags for a shard: the prior stays with rank 0 only."""
    return flags if rank == 0 else (flags | GLM_FLAG_NO_PRIOR)


def allreduce_sum_(f, g, group=None) -> None:
    """Sum the shards' f (FP64) and g in place over the process group: the
    only exchange of a sharded evaluation."""
    import torch.distributed as dist
    dist.all_reduce(f, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
