"""Screen-space split of one frame over several renderers: the sort-middle form of the
pipeline (Sec. 2, "Pipeline description": the screen is cut into bins that are rasterised
independently of one another once binning has sorted the quads into them).

Every renderer runs setup and binning on all quads of the frame, then depth-sorts and
rasterises only the 32x32-pixel tiles it owns (lr_view.owned_tiles); the tiles are disjoint,
so the only exchange is one gather of the owned tiles into the full frame. Splitting by quad
subsets instead (sort-last) would not be exact without exchanging whole per-pixel fragment
lists, so it is not offered.

Host logic only: which rank owns which tile, each rank's owned-tile bit set and tile
rectangles, and the gather of the tiles over torch.distributed (NCCL for device tensors,
gloo for host tensors). Nothing here computes pixels.
"""
from __future__ import annotations

import numpy as np

TILE = 32


def tile_grid(width: int, height: int) -> tuple[int, int]:
    """Tiles per row and per column of a width x height frame."""
    return (width + TILE - 1) // TILE, (height + TILE - 1) // TILE


def assign_tiles(width: int, height: int, world: int, costs=None) -> np.ndarray:
    """owner[ty][tx]: the rank that rasterises each tile.

    costs None: diagonal interleaving, owner = (tx + ty) mod world, which spreads any
    smooth density (a dense centre, a dense band) evenly over the ranks.
    costs: an estimate of each tile's raster work, float[nty][ntx] (e.g. the previous
    frame's bin reference counts or fragment counts): tiles are taken in decreasing cost
    and each goes to the rank with the least work so far (longest processing time first),
    ties to the lower rank, so that the most loaded rank exceeds the mean by at most one
    tile's cost.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    ntx, nty = tile_grid(width, height)
    if costs is None:
        ty, tx = np.meshgrid(np.arange(nty), np.arange(ntx), indexing="ij")
        return ((tx + ty) % world).astype(np.int32)
    c = np.asarray(costs, np.float64)
    if c.shape != (nty, ntx):
        raise ValueError(f"costs must have shape {(nty, ntx)}")
    owner = np.zeros(nty * ntx, np.int32)
    load = np.zeros(world, np.float64)
    for t in np.argsort(-c.reshape(-1), kind="stable"):
        r = int(np.argmin(load))
        owner[t] = r
        load[r] += c.reshape(-1)[t]
    return owner.reshape(nty, ntx)


def owned_bitset(owner: np.ndarray, rank: int) -> np.ndarray:
    """The owned-tile bit set of one rank in the layout lr_view.owned_tiles takes: tile t
    (row-major) is bit t % 32 of word t // 32."""
    flat = (np.asarray(owner).reshape(-1) == rank)
    words = np.zeros((flat.size + 31) // 32, np.uint32)
    idx = np.nonzero(flat)[0]
    np.bitwise_or.at(words, idx // 32, (np.uint32(1) << (idx % 32).astype(np.uint32)))
    return words


def tile_rects(owner: np.ndarray, rank: int, width: int, height: int):
    """Pixel rectangles (x0, y0, x1, y1), end-exclusive and clipped to the frame, of the
    tiles a rank owns, in row-major tile order."""
    out = []
    nty, ntx = owner.shape
    for ty in range(nty):
        for tx in range(ntx):
            if owner[ty, tx] == rank:
                out.append((tx * TILE, ty * TILE, min((tx + 1) * TILE, width), min((ty + 1) * TILE, height)))
    return out


def pack_tiles(frame, owner: np.ndarray, rank: int, capacity: int | None = None):
    """The owned tiles of frame [H][W][C] (a torch tensor) as one tensor
    [capacity][32][32][C], row-major tile order, tiles at the frame's edge zero-padded, and
    rows past the rank's tile count zero."""
    import torch
    H, W = frame.shape[0], frame.shape[1]
    rects = tile_rects(owner, rank, W, H)
    n = len(rects) if capacity is None else capacity
    out = torch.zeros((n, TILE, TILE) + tuple(frame.shape[2:]), dtype=frame.dtype, device=frame.device)
    for i, (x0, y0, x1, y1) in enumerate(rects):
        out[i, : y1 - y0, : x1 - x0] = frame[y0:y1, x0:x1]
    return out


def unpack_tiles(frame, tiles, owner: np.ndarray, rank: int):
    """Writes a rank's packed tiles (pack_tiles' layout) into frame [H][W][C]."""
    H, W = frame.shape[0], frame.shape[1]
    for i, (x0, y0, x1, y1) in enumerate(tile_rects(owner, rank, W, H)):
        frame[y0:y1, x0:x1] = tiles[i, : y1 - y0, : x1 - x0]
    return frame


def gather_frame(local, owner: np.ndarray, dist=None):
    """The full frame on every rank from each rank's frame, in which only its owned tiles
    are valid: one all_gather of the packed tiles (padded to the largest tile count), then
    every rank's tiles written into a copy of its own frame. Without a process group (one
    rank) the frame is returned as it is."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local
    world, rank = dist.get_world_size(), dist.get_rank()
    cap = max(int((owner == r).sum()) for r in range(world))
    mine = pack_tiles(local, owner, rank, cap)
    parts = [mine.new_empty(mine.shape) for _ in range(world)]
    dist.all_gather(parts, mine)
    out = local.clone()
    for r in range(world):
        if r != rank:
            unpack_tiles(out, parts[r], owner, r)
    return out
