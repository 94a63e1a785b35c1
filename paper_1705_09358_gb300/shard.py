"""Multi-device form: shard the split frontier across ranks, sum four counters.

Subtrees below the breadth-first split are independent, so rank r of R
searches only the frontier frames whose index is r modulo R (the engine's
``shard_index`` / ``shard_count`` options); counters above the frontier are
counted by rank 0 alone.  The one exchange step is a wrapping 64-bit sum of
(matches, states, nodes, hash) over the ranks, which gives the unsharded
result bit for bit.
"""
from __future__ import annotations

KEYS = ("matches", "states", "nodes", "hash")
_MASK = (1 << 64) - 1


def _to_i64(x: int) -> int:
    x &= _MASK
    return x - (1 << 64) if x >= (1 << 63) else x


def reduce_counters(local: dict, group=None) -> dict:
    """Sum the four counters over the process group (mod 2^64).

    int64 addition wraps like uint64 addition, so the bit pattern of the sum
    is the unsigned sum modulo 2^64.
    """
    import torch
    import torch.distributed as dist
    backend = dist.get_backend(group)
    device = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([_to_i64(int(local[k])) for k in KEYS], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return {k: int(v) & _MASK for k, v in zip(KEYS, t.cpu().tolist())}


def count_sharded(count_fn, rank: int, world: int, split_depth: int = 0, group=None) -> dict:
    """Run this rank's shard with ``count_fn(shard_index=, shard_count=,
    split_depth=)`` (returning a dict with the four counters) and reduce."""
    local = count_fn(shard_index=rank, shard_count=world, split_depth=split_depth)
    return reduce_counters(local, group)
