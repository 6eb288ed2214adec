"""The 8x8-block rasteriser (lr_config.block_h = 8) against the oracle: counts and coverage
hashes bit-exact, colour within 1e-5, for flat and per-vertex colours, every sorter capacity
it is built for, every bin size, dense and ragged scenes, the full 1080p frames, owned-tile
sets; its exact-path mask equals the 8x4 kernel's (the same pixels take the exact path, so
the backward pass can use it)."""
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


def _render(lr, s, k=3, bin_size=32, block_h=8, carry=False, owned=None, out=None, mask=False):
    r = lr.Renderer(sorter_k=k, bin_size=bin_size, block_h=block_h, carry_colors=carry)
    if out is None:
        out = r.make_outputs(s.width, s.height, rgba8=True, count=True, hash=True, exact_mask=mask)
    r.render(lr.DeviceScene.from_scene(s), s.width, s.height, owned_tiles=owned, out=out)
    torch.cuda.synchronize()
    st = r.stats()
    r.close()
    return out, st


def _compare(out, st, o, sel=None):
    sel = np.ones(o["count"].shape, bool) if sel is None else sel
    np.testing.assert_array_equal(out["count"].cpu().numpy().view(np.uint32)[sel], o["count"][sel])
    np.testing.assert_array_equal(out["hash"].cpu().numpy().view(np.uint64)[sel], o["hash"][sel])
    d = np.abs(out["rgba"].cpu().numpy()[sel].astype(np.float64) - o["rgba"][sel]).max()
    assert d <= COLOR_TOL, d
    d8 = np.abs(out["rgba8"].cpu().numpy()[sel].astype(np.int32) - o["rgba8"][sel].astype(np.int32)).max()
    assert d8 <= 1
    if st is not None:
        assert st["fragments"] == int(o["count"][sel].sum())


def _scenes():
    return {
        "frustum256": scenegen.config_small_frustum(),
        "frustum_ragged": scenegen.frustum_parallelograms(3000, 200, 141, seed=4),
        "layers_vertex": scenegen.wavy_layers(333, 190, layers=32, nx=48, ny=24, seed=1),
        "layers_flat": scenegen.wavy_layers(256, 256, layers=24, nx=32, ny=32, seed=2, color_mode=scenegen.COLOR_FLAT),
        "particles": scenegen.gaussian_particles(60_000, 320, 180, seed=3),
        "big_near_quads": scenegen.frustum_parallelograms(300, 160, 96, seed=9, edge_range=(0.5, 6.0), far=8.0),
        "tiny": scenegen.frustum_parallelograms(40, 13, 7, seed=2, edge_range=(0.5, 3.0), far=10.0),
    }


@pytest.mark.parametrize("name", list(_scenes()))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_blocks_match_oracle(lr, name, k):
    s = _scenes()[name]
    out, st = _render(lr, s, k)
    assert st["status"] == 0
    _compare(out, st, oracle.render(s))


@pytest.mark.parametrize("bin_size", [16, 64])
@pytest.mark.parametrize("name", ["layers_vertex", "particles", "frustum_ragged"])
def test_blocks_every_bin_size(lr, bin_size, name):
    s = _scenes()[name]
    out, st = _render(lr, s, 1, bin_size=bin_size)
    _compare(out, st, oracle.render(s))


def test_blocks_carried_flat_colours(lr):
    s = _scenes()["particles"]
    out, st = _render(lr, s, 1, carry=True)
    _compare(out, st, oracle.render(s))


@pytest.mark.parametrize("name", ["layers", "particles"])
def test_blocks_full_size(lr, name):
    s = {"layers": scenegen.config_layers_1080p, "particles": scenegen.config_particles_1080p}[name]()
    out, st = _render(lr, s, 1)
    assert st["status"] == 0
    _compare(out, st, oracle.render(s))


def test_blocks_exact_mask_equals_half_blocks(lr):
    s = _scenes()["layers_vertex"]
    a, sa = _render(lr, s, 1, block_h=8, mask=True)
    b, sb = _render(lr, s, 1, block_h=4, mask=True)
    assert sa["overflow_pixels"] == sb["overflow_pixels"] > 0
    assert torch.equal(a["exact_mask"], b["exact_mask"])
    assert torch.equal(a["count"], b["count"]) and torch.equal(a["hash"], b["hash"])


def test_blocks_with_owned_tiles(lr):
    s = _scenes()["layers_vertex"]
    o = oracle.render(s)
    owner = PT.assign_tiles(s.width, s.height, 2)
    for rank in range(2):
        bits = torch.from_numpy(PT.owned_bitset(owner, rank).view(np.int32)).cuda()
        r = lr.Renderer(sorter_k=1, block_h=8)
        out = r.make_outputs(s.width, s.height, rgba8=True, count=True, hash=True)
        out["rgba"].fill_(float("nan"))
        r.render(lr.DeviceScene.from_scene(s), s.width, s.height, owned_tiles=bits, out=out)
        torch.cuda.synchronize()
        r.close()
        mine = np.zeros((s.height, s.width), bool)
        for x0, y0, x1, y1 in PT.tile_rects(owner, rank, s.width, s.height):
            mine[y0:y1, x0:x1] = True
        _compare(out, None, o, mine)
        assert np.isnan(out["rgba"].cpu().numpy()[~mine]).all()


def test_blocks_fall_back_where_not_built(lr):
    # K = 8, the alpha threshold and lit colours take the 8x4 kernel on a block_h = 8 context
    s = _scenes()["layers_vertex"]
    out, st = _render(lr, s, 8)
    _compare(out, st, oracle.render(s))
    r = lr.Renderer(sorter_k=1, block_h=8, alpha_threshold=True)
    a = r.render(lr.DeviceScene.from_scene(s), s.width, s.height)
    torch.cuda.synchronize()
    ref = oracle.render_threshold(s)
    assert np.abs(a["rgba"].cpu().numpy().astype(np.float64) - ref["rgba"]).max() <= COLOR_TOL
    r.close()
