"""Sharding one migration over processes by frequency.

Every frequency line is extrapolated through all depth steps without reference
to any other frequency (Sec. II: the frequencies decouple in the f-x domain),
so ranks can own disjoint, contiguous blocks of the band with no
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


def _image_shape(d):
    """[nz][nx] for a 2-D description, [nz][ny][nx] for a 3-D one."""
    return (d.nz, d.ny, d.nx) if hasattr(d, "ny") else (d.nz, d.nx)


def _migrate3d_on_device(sd, slab, vel, table, launch=None, stream=None):
    """One rank's block of a 3-D problem through the library (all depth rows
    of `sd`), then its image (float32 [nz][ny][nx])."""
    import torch

    import paper_1912_05529_gb300 as fx
    dev = slab.device
    partials = torch.empty((fx.fxmig3d_num_partials(sd), sd.nz, sd.ny, sd.nx), dtype=torch.float32, device=dev)
    ws = torch.zeros(fx.fxmig3d_workspace_bytes(sd), dtype=torch.uint8, device=dev)
    image = torch.empty((sd.nz, sd.ny, sd.nx), dtype=torch.float32, device=dev)
    fx.fxmig3d_migrate(sd, slab, vel, table, partials, 0, sd.nz, ws, stream=stream)
    fx.fxmig3d_image(sd, partials, image, stream)
    rc = fx.fxmig_check(ws, stream)
    if rc != fx.FXMIG_OK:
        raise fx.FxmigError(rc, "fxmig3d_migrate (frequency shard)")
    return image


def _migrate_on_device(sd, slab, vel, table, launch=None, stream=None):
    """One rank's block through the library: the depth loop over all rows of
    `sd` on the rank's lines, then its image (float32 [nz][nx], on the
    slab's device)."""
    import torch

    import paper_1912_05529_gb300 as fx
    dev = slab.device
    partials = torch.empty((fx.fxmig_num_partials(sd, launch), sd.nz, sd.nx), dtype=torch.float32, device=dev)
    ws = torch.zeros(fx.fxmig_workspace_bytes(sd, fx.FXMIG_WS_MIGRATE), dtype=torch.uint8, device=dev)
    image = torch.empty((sd.nz, sd.nx), dtype=torch.float32, device=dev)
    fx.fxmig_migrate_ex(sd, launch, slab, vel, table, partials, 0, sd.nz, ws, stream)
    fx.fxmig_image(sd, partials, image, stream)
    rc = fx.fxmig_check(ws, stream)
    if rc != fx.FXMIG_OK:
        raise fx.FxmigError(rc, "fxmig_migrate_ex (frequency shard)")
    return image


def migrate_frequency_shard(d, slab, vel, table, launch=None, group=None, stream=None, migrate_fn=None):
    """Algorithm 1 over a frequency-sharded band: this rank migrates its
    contiguous block of lines (frequency_block / shard_desc: same table range
    k_max, first bin i0 + j0) and the images of all ranks are summed in rank
    order on every rank.

    slab       this rank's lines [j0, j0 + n) of the band, [n][nx] complex64,
               or for a 3-D description (Desc3d) its planes [n][ny][nx]
               (device tensor; ignored when the block is empty)
    vel, table the full velocity field and operator table (every rank)
    migrate_fn (sd, slab, vel, table, launch, stream) -> image [nz][nx] (3-D:
               [nz][ny][nx]); the library by default
    Returns the image of the whole band (same on every rank)."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    sd = shard_desc(d, world, rank)
    if sd is None:
        dev = vel.device if hasattr(vel, "device") else "cpu"
        image = torch.zeros(_image_shape(d), dtype=torch.float64 if migrate_fn else torch.float32, device=dev)
    else:
        default = _migrate3d_on_device if hasattr(d, "ny") else _migrate_on_device
        image = (migrate_fn or default)(sd, slab, vel, table, launch, stream)
    return reduce_images_rank_order(image, group)
