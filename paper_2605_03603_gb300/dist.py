"""Combining sharded counts across ranks (one process per GPU).

Algorithm 2 treats every anchor of the anchor side on its own, so a count whose
anchors are split over ranks (``sbc_count_ex(..., shard=r, shard_count=N)``)
is the exact sum of the ranks' partial counts. Partials are unsigned 128-bit
integers; they are summed exactly as four 32-bit limbs held in int64 (a limb
sum stays below 2^63 for up to 2^31 ranks) and carried on the host. The sum of
the partials of a count that fits in 128 bits fits in 128 bits; a larger sum
raises OverflowError, as the single-GPU path does.

Works with any torch.distributed backend that sums int64 tensors (gloo on CPU
tensors, nccl on CUDA tensors); the caller passes the device its backend needs.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

LIMBS = 4
_MASK32 = (1 << 32) - 1
U128_MAX = (1 << 128) - 1


def to_limbs(x: int) -> list[int]:
    """Four little-endian 32-bit limbs of an unsigned 128-bit integer."""
    if not 0 <= x <= U128_MAX:
        raise OverflowError(f"{x} is not an unsigned 128-bit value")
    return [(x >> (32 * i)) & _MASK32 for i in range(LIMBS)]


def from_limbs(limbs) -> int:
    """Value of little-endian limbs (any size each: carries are propagated)."""
    return sum(int(v) << (32 * i) for i, v in enumerate(limbs))


def allreduce_counts(values, group=None, device=None) -> list[int]:
    """Exact sums over all ranks of each entry of `values` (u128 integers).

    Every rank passes the same number of values; every rank gets the sums."""
    vals = [int(v) for v in values]
    flat = [limb for v in vals for limb in to_limbs(v)]
    t = torch.tensor(flat if flat else [0], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    host = t.cpu().tolist()
    out = []
    for i in range(len(vals)):
        s = from_limbs(host[LIMBS * i:LIMBS * (i + 1)])
        if s > U128_MAX:
            raise OverflowError("sharded count exceeds 128 bits")
        out.append(s)
    return out


def max_over_ranks(x: float, group=None, device=None) -> float:
    """The largest of the ranks' values (step times are the slowest rank's)."""
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
