"""Range sharding of one exponential sum across ranks.

The 2^k Gray-code indices split into disjoint contiguous ranges; each rank
sums its own range (on its GPU) and the raw partials, exact integers modulo
2^64 over the common sqrt2^e0, are gathered (40 bytes per rank) and added with
zxp_zomega_add.  Integer addition makes the result independent of the number
of ranks and of the order of the partials.
"""
from __future__ import annotations

from typing import Callable, Sequence, Tuple

from . import zxp_zomega_add, zxp_zomega_canon

Partial = Tuple[int, int, int, int, int]


def shard_range(k: int, world: int, rank: int) -> Tuple[int, int]:
    """[first, first + count) of rank `rank` among `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world / rank")
    total = 1 << k
    base, rem = divmod(total, world)
    first = rank * base + min(rank, rem)
    return first, base + (1 if rank < rem else 0)


def combine(partials: Sequence[Partial]) -> Partial:
    """Exact sum of raw partials (any order)."""
    acc = None
    for p in partials:
        acc = tuple(p) if acc is None else zxp_zomega_add(acc, p)
    return acc


def sharded_sum(eval_range: Callable[[int, int], Partial], k: int, group=None,
                canonical: bool = True) -> Partial:
    """Sum over [0, 2^k) split across the ranks of `group` (torch.distributed).

    eval_range(first, count) returns this rank's raw partial (for example
    zxp_eval on the rank's own GPU).  The partials are all-gathered as int64
    tensors on the group's device and combined exactly on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    first, count = shard_range(k, world, rank)
    mine = eval_range(first, count)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([_i64(v) for v in mine], dtype=torch.int64, device=dev)
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    total = combine([tuple(int(v) for v in o.tolist()) for o in out])
    return zxp_zomega_canon(total) if canonical else total


def _i64(v: int) -> int:
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >> 63 else v
