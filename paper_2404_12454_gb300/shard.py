"""One field spread over several GPUs by detector rows.

The plane-evaluation method is pixel-parallel (Sec. 5): every pixel sums every beamlet, and
no pixel needs another's value.  So the field of one (beamlet table, detector) pair shards
by pixels with the beamlet table replicated: rank r evaluates a contiguous slab of detector
rows through ``gbd_field_rows`` (which gives the same bits as those rows of the whole-
detector ``gbd_field``), and one all-gather assembles the field.  The gather is the only
exchange; nothing crosses GPUs while the kernels run.

This module holds the partition and the gather bookkeeping (no arithmetic of the method);
``torch.distributed`` carries the gather (NCCL between GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

from typing import Callable, List, Tuple


def slab_bounds(ny: int, world: int, rank: int) -> Tuple[int, int]:
    """Rows [r0, r1) of rank ``rank`` out of ``world``: contiguous, in rank order, sizes
    differing by at most one row (ranks beyond ny get empty slabs)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if ny < 0:
        raise ValueError("ny must be >= 0")
    return rank * ny // world, (rank + 1) * ny // world


def all_slabs(ny: int, world: int) -> List[Tuple[int, int]]:
    return [slab_bounds(ny, world, r) for r in range(world)]


def gather_rows(local, ny: int, group=None):
    """All-gather of each rank's slab (``local``: [r1 - r0, nx] complex tensor of this
    rank's rows) into the whole [ny, nx] field on every rank.  Slabs are padded to the
    largest slab's rows for the collective (which needs equal sizes) and cut back."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    r0, r1 = slab_bounds(ny, world, rank)
    if local.shape[0] != r1 - r0:
        raise ValueError(f"rank {rank} holds {local.shape[0]} rows, its slab has {r1 - r0}")
    nx = local.shape[1]
    rows_max = max(b - a for a, b in all_slabs(ny, world))
    # complex tensors travel as their real view (gloo has no complex reductions or gathers)
    real = torch.view_as_real(local.contiguous())
    send = torch.zeros((rows_max, nx, 2), dtype=real.dtype, device=real.device)
    send[: r1 - r0] = real
    recv = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    parts = [recv[r][: b - a] for r, (a, b) in enumerate(all_slabs(ny, world))]
    return torch.view_as_complex(torch.cat(parts, dim=0).contiguous())


def field_sharded(beamlets, wavelength: float, detector, precision: int, group=None,
                  stream=None, slab_fn: Callable = None):
    """The whole field on every rank, each rank computing its own slab of rows.

    ``slab_fn(beamlets, wavelength, detector, r0, r1, precision, stream)`` evaluates rows
    [r0, r1); by default the library's ``gbd.field_rows``."""
    import torch.distributed as dist

    if slab_fn is None:
        from . import gbd

        def slab_fn(b, lam, det, r0, r1, prec, s):
            return gbd.field_rows(b, lam, det, r0, r1, prec, stream=s)

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    r0, r1 = slab_bounds(detector.ny, world, rank)
    local = slab_fn(beamlets, wavelength, detector, r0, r1, precision, stream)
    return gather_rows(local, detector.ny, group)
