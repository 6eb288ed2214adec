"""The screen-space split of one frame on one GPU: each rank's render with its owned-tile
set (lr_view.owned_tiles) writes exactly its tiles, those match the oracle (counts and
hashes bit-exact, colour within 1e-5), everything else is left untouched, and the tiles of
all ranks gathered form the oracle's frame. Ranks run one after another here (one GPU);
the exchange itself is tested on CPU ranks."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2405_13364_gb300 import partition as PT

pytestmark = pytest.mark.gpu

COLOR_TOL = 1e-5


@pytest.fixture(scope="module")
def lr():
    import paper_2405_13364_gb300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    P.load_library()
    return P


def _sentinel_outputs(r, W, H):
    out = r.make_outputs(W, H, rgba8=True, count=True, hash=True)
    out["rgba"].fill_(float("nan"))
    out["rgba8"].fill_(7)
    out["count"].fill_(-1)
    out["hash"].fill_(-1)
    return out


def _owned_pixels(owner, rank, W, H):
    m = np.zeros((H, W), bool)
    for x0, y0, x1, y1 in PT.tile_rects(owner, rank, W, H):
        m[y0:y1, x0:x1] = True
    return m


def _check_split(lr, scene, world, costs=None, k=3):
    W, H = scene.width, scene.height
    o = oracle.render(scene)
    owner = PT.assign_tiles(W, H, world, costs)
    r = lr.Renderer(sorter_k=k)
    ds = lr.DeviceScene.from_scene(scene)
    full = {k_: None for k_ in ("rgba", "count", "hash")}
    frags = 0
    for rank in range(world):
        bits = torch.from_numpy(PT.owned_bitset(owner, rank).view(np.int32)).cuda()
        out = _sentinel_outputs(r, W, H)
        r.render(ds, W, H, owned_tiles=bits, out=out)
        torch.cuda.synchronize()
        st = r.stats()
        assert st["status"] == 0
        frags += st["fragments"]
        mine = _owned_pixels(owner, rank, W, H)
        rgba = out["rgba"].cpu().numpy()
        cnt = out["count"].cpu().numpy().view(np.uint32)
        hsh = out["hash"].cpu().numpy().view(np.uint64)
        # the owned tiles match the oracle
        np.testing.assert_array_equal(cnt[mine], o["count"][mine])
        np.testing.assert_array_equal(hsh[mine], o["hash"][mine])
        assert np.abs(rgba[mine].astype(np.float64) - o["rgba"][mine]).max() <= COLOR_TOL
        assert st["fragments"] == int(o["count"][mine].sum())
        # the others are untouched
        assert np.isnan(rgba[~mine]).all()
        assert np.all(cnt[~mine] == 0xFFFFFFFF) and np.all(out["rgba8"].cpu().numpy()[~mine] == 7)
        # gather (on one GPU: the tiles of every rank written into one frame)
        for key in full:
            if full[key] is None:
                full[key] = out[key].clone()
            else:
                PT.unpack_tiles(full[key], PT.pack_tiles(out[key], owner, rank), owner, rank)
    np.testing.assert_array_equal(full["count"].cpu().numpy().view(np.uint32), o["count"])
    np.testing.assert_array_equal(full["hash"].cpu().numpy().view(np.uint64), o["hash"])
    assert np.abs(full["rgba"].cpu().numpy().astype(np.float64) - o["rgba"]).max() <= COLOR_TOL
    assert frags == o["stats"]["fragments"]
    r.close()


@pytest.mark.parametrize("world", [2, 3])
def test_split_layers(lr, world):
    _check_split(lr, scenegen.wavy_layers(333, 190, layers=32, nx=48, ny=24, seed=1), world, k=1)


def test_split_particles_cost_balanced(lr):
    s = scenegen.gaussian_particles(60_000, 320, 180, seed=3)
    # per-tile cost: the oracle's fragments per tile (as a previous frame would give)
    cnt = oracle.render(s)["count"].astype(np.float64)
    ntx, nty = PT.tile_grid(s.width, s.height)
    pad = np.zeros((nty * 32, ntx * 32))
    pad[: s.height, : s.width] = cnt
    costs = pad.reshape(nty, 32, ntx, 32).sum((1, 3))
    _check_split(lr, s, 4, costs)


def test_split_full_size_layers(lr):
    _check_split(lr, scenegen.config_layers_1080p(), 2, k=1)


def test_owned_tiles_in_a_batch(lr):
    # two views of one batch with different owned sets, against single-view renders
    s = scenegen.config_small_frustum()
    W, H = s.width, s.height
    r = lr.Renderer(sorter_k=3)
    ds = lr.DeviceScene.from_scene(s)
    owner = PT.assign_tiles(W, H, 2)
    outs, views = [], []
    for rank in range(2):
        bits = torch.from_numpy(PT.owned_bitset(owner, rank).view(np.int32)).cuda()
        out = _sentinel_outputs(r, W, H)
        outs.append((out, bits))
        views.append(r.view_struct(ds, W, H, out, bits))
    r.render_views(views)
    torch.cuda.synchronize()
    ref = r.render(ds, W, H, count=True)
    torch.cuda.synchronize()
    for rank, (out, _) in enumerate(outs):
        mine = torch.from_numpy(_owned_pixels(owner, rank, W, H)).cuda()
        assert torch.equal(out["count"][mine], ref["count"][mine])
        assert torch.equal(out["rgba"][mine], ref["rgba"][mine])
        assert torch.isnan(out["rgba"][~mine]).all()
    r.close()
