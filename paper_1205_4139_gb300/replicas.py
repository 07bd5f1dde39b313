"""Replica split of a batch of independent recovery instances over ranks.

OMP instances are independent (each solves Algorithm 1.1 on its own
measurement), so one process per GPU solves its own share of the batch and no
data crosses between ranks: weak scaling with a fixed per-rank batch.  The
only collective is the timing reduction (the slowest rank's time bounds the
job).  Instance seeds follow the synthetic generator's convention (instance
g of a batch is drawn from seed + 1 + g), so rank r's share of a global batch
of world * B instances is the contiguous block [r B, (r + 1) B).
"""
from __future__ import annotations


def shard(rank: int, world: int, per_rank: int) -> range:
    """Global instance indices rank `rank` solves (contiguous, disjoint over
    ranks, covering [0, world * per_rank))."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("need 0 <= rank < world and per_rank >= 0")
    return range(rank * per_rank, (rank + 1) * per_rank)


def shard_seed(rank: int, per_rank: int, base_seed: int = 0) -> int:
    """Seed that makes the generator's instance b of this rank equal instance
    rank * per_rank + b of the global batch drawn with `base_seed`."""
    return base_seed + rank * per_rank


def max_over_ranks(values, device=None) -> list[float]:
    """Element-wise maximum of a list of floats over all ranks of the default
    process group (the values themselves when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def argmax_over_ranks(value: float, index: int, device=None) -> tuple[float, int]:
    """Identification across ranks that each hold a slice of the output index
    j (one instance sharded by j): every rank passes its slice's largest
    |h(j)|^2 and the lowest j that reaches it (-1 and a negative value when
    its slice has no candidate); every rank gets the overall largest value
    and the lowest j among the ranks that reach it (Algorithm 1.1 step 3 with
    the ties to the lower index).  Two small all-reduces: MAX of the values,
    then MIN of the indices of the ranks at that value."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value), int(index)
    v = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    best = float(v.item())
    big = 2 ** 62
    j = torch.tensor([int(index) if (index >= 0 and float(value) == best) else big], dtype=torch.int64, device=device)
    dist.all_reduce(j, op=dist.ReduceOp.MIN)
    jj = int(j.item())
    return best, (-1 if jj == big else jj)
