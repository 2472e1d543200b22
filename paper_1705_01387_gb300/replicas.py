"""Replica parallelism over independent random vectors.

The stochastic trace (Sec. 3.1, Eq. 13) averages over independent random
vectors, and each vector's Chebyshev moments are computed without reference to
any other (the paper runs them one after another, or as separate jobs).  Ranks
therefore each take a contiguous share of the vector indices; nothing moves
between ranks while moments are computed.  The only exchange is the final
average of the moment arrays (one all-reduce of R*Nt*M doubles) and the maximum
of the ranks' wall times for reporting.
"""
from __future__ import annotations


def shard_vectors(total: int, world: int, rank: int) -> tuple[int, int]:
    """(first_vector, count) of rank `rank` when `total` vectors are split over
    `world` ranks as evenly as possible (earlier ranks take the remainder)."""
    if world <= 0 or not (0 <= rank < world) or total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def average_moments(local_sum, local_count: int, group=None):
    """Average of moment arrays over all ranks' vectors: all-reduce (SUM) of the
    local sums and counts, then divide.  `local_sum` is a float64 torch tensor
    holding the sum over this rank's vectors; returns the global mean."""
    import torch
    import torch.distributed as dist
    cnt = torch.tensor([float(local_count)], dtype=torch.float64, device=local_sum.device)
    tot = local_sum.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM, group=group)
    return tot / cnt


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
