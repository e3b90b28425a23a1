"""Whole-frame regions split by pixels across ranks (one process per GPU).

Pixel and block regions shard with no exchange (each rank owns whole
regions).  A whole-frame region cannot: every rank holds a band of rows of each
training frame, and a frame's tree (Alg. 1) holds a leaf when any pixel of the
whole frame reaches it.  So the path has one exchange step here: each rank
takes its band's per-frame leaf sets (``ocq_occupancy``), the ranks gather
them (``torch.distributed.all_gather``, 8^d/8 bytes per frame and rank), and
``ocq_merge_occupancy`` unions them per frame and keeps the leaves held by at
least T frames (Alg. 2).  Every rank then holds the same model and classifies
its own band of each test frame (Alg. 3).  This module is host plumbing only:
the leaf sets, their union and the count are computed by the CUDA library.
"""
from __future__ import annotations

from . import ocq

FRAME = ocq.OCQ_REGION_FRAME


def frame_band(H: int, rank: int, world: int):
    """Rows [y0, y1) of an H-row frame that ``rank`` of ``world`` holds: bands
    as equal as possible, the first H % world ranks one row taller."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(H, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def gather_parts(local, group=None):
    """All ranks' tensors of the same shape, stacked rank-major ([world, ...])."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local.contiguous(), group=group)
    return torch.stack(parts)


def build_model_banded(band, H: int, depth: int, T: int, group=None, stream=None):
    """The whole-frame model of N training frames of which this rank holds the
    row band ``band`` (CUDA uint8 [N, h, W, 3], h = the band's rows; bands as
    ``frame_band`` gives them).  Collective: every rank of ``group`` calls it
    with its own band; each gets the same model."""
    import torch

    N, h, W, _ = band.shape
    wpr = 1 if depth <= 2 else 1 << (3 * depth - 6)
    occ = torch.empty((N, 1, wpr), dtype=torch.int64, device=band.device)
    if h > 0:
        ocq.ocq_occupancy(band.contiguous(), N, h, W, FRAME, 0, depth, occ, stream)
    else:
        occ.zero_()  # a rank without rows holds no pixels: empty leaf sets
    parts = gather_parts(occ, group)
    return ocq.ocq_merge_occupancy(parts, parts.shape[0], N, H, W, FRAME, 0, depth, T, stream)
