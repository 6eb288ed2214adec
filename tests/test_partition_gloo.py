"""Host logic of the screen-space split of one frame (sort-middle form), on CPU: tile
ownership, owned-tile bit sets, tile rectangles, and the all_gather of tiles over two gloo
ranks (each rank holds valid pixels only in its own tiles)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2405_13364_gb300 import partition as PT


@pytest.mark.parametrize("wh", [(1920, 1080), (256, 256), (200, 141), (31, 17)])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_every_tile_owned_once_and_rects_cover_the_frame(wh, world):
    W, H = wh
    owner = PT.assign_tiles(W, H, world)
    ntx, nty = PT.tile_grid(W, H)
    assert owner.shape == (nty, ntx) and owner.min() >= 0 and owner.max() < world
    cover = np.zeros((H, W), np.int32)
    words = [PT.owned_bitset(owner, r) for r in range(world)]
    for r in range(world):
        for x0, y0, x1, y1 in PT.tile_rects(owner, r, W, H):
            assert 0 <= x0 < x1 <= W and 0 <= y0 < y1 <= H
            cover[y0:y1, x0:x1] += 1
    assert np.all(cover == 1)
    # the bit sets partition the tiles too
    t = np.arange(ntx * nty)
    bits = np.stack([(w[t // 32] >> (t % 32).astype(np.uint32)) & 1 for w in words])
    assert np.all(bits.sum(0) == 1)
    assert np.all(bits.argmax(0) == owner.reshape(-1))


def test_cost_balanced_assignment():
    rng = np.random.default_rng(0)
    W, H = 1920, 1080
    ntx, nty = PT.tile_grid(W, H)
    ty, tx = np.meshgrid(np.arange(nty), np.arange(ntx), indexing="ij")
    # a dense centre, as in the particle workload
    costs = 1e4 * np.exp(-(((tx - ntx / 2) / 8.0) ** 2 + ((ty - nty / 2) / 6.0) ** 2)) + rng.random((nty, ntx))
    for world in (2, 4, 8):
        owner = PT.assign_tiles(W, H, world, costs)
        load = np.array([costs[owner == r].sum() for r in range(world)])
        assert load.max() <= costs.sum() / world + costs.max() + 1e-6
        assert np.all(np.bincount(owner.reshape(-1), minlength=world) > 0)


def test_pack_unpack_roundtrip():
    W, H = 100, 70
    img = torch.arange(H * W * 4, dtype=torch.float32).reshape(H, W, 4)
    owner = PT.assign_tiles(W, H, 3)
    out = torch.full_like(img, -1.0)
    for r in range(3):
        PT.unpack_tiles(out, PT.pack_tiles(img, owner, r), owner, r)
    assert torch.equal(out, img)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    W, H = 200, 141
    g = torch.Generator().manual_seed(5)
    ref = torch.rand((H, W, 4), generator=g)              # the same reference on every rank
    owner = PT.assign_tiles(W, H, world)
    # this rank's frame: valid in its own tiles, garbage elsewhere
    local = torch.full((H, W, 4), float(100 + rank))
    for x0, y0, x1, y1 in PT.tile_rects(owner, rank, W, H):
        local[y0:y1, x0:x1] = ref[y0:y1, x0:x1]
    full = PT.gather_frame(local, owner, dist)
    ok = bool(torch.equal(full, ref))
    res = [None] * world
    dist.all_gather_object(res, ok)
    if rank == 0:
        q.put(res)
    dist.destroy_process_group()


def test_gather_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [True, True]


def test_gather_single_rank_is_identity():
    img = torch.rand(40, 50, 4)
    owner = PT.assign_tiles(50, 40, 1)
    assert PT.gather_frame(img, owner, None) is img
