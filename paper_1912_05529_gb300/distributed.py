"""Sharding one migration over processes by frequency.

Every frequency line is extrapolated independently through all depth steps
(Sec. II: the extrapolation "can be performed independently for each
frequency"), so ranks can own disjoint, contiguous blocks of the band with no
communication until the end; the only exchange is the image, the sum over
frequencies (Algorithm 1), which is reduced here in rank order so that the
result does not depend on the collective's internal order.
"""
from __future__ import annotations

import ctypes


def frequency_block(nw: int, world: int, rank: int) -> tuple[int, int]:
    """(first line, line count) of `rank`'s contiguous block of nw lines;
    block sizes differ by at most one, lower ranks get the larger ones."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(nw, world)
    j0 = rank * base + min(rank, extra)
    return j0, base + (1 if rank < extra else 0)


def shard_desc(d, world: int, rank: int):
    """Descriptor of `rank`'s frequency block (same table range k_max), or None
    when the block is empty."""
    j0, n = frequency_block(d.nw, world, rank)
    if n == 0:
        return None
    s = type(d)()
    ctypes.pointer(s)[0] = d
    s.i0 = d.i0 + j0
    s.nw = n
    return s


def reduce_images_rank_order(image, group=None):
    """Sum of every rank's partial image, added in ascending rank order on
    every rank (all-gather, then a fixed-order sum)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(image) for _ in range(world)]
    dist.all_gather(parts, image.contiguous(), group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out
