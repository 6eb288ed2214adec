"""The strip rasteriser (lr_config.shared_setup = 1: a CTA sets each candidate triangle up
once per 32x8 strip of a bin) against the oracle: counts and coverage hashes bit-exact,
colour within 1e-5, for flat, carried and per-vertex colours, every sorter capacity it is
built for, dense and ragged scenes, the full 1080p frames and owned-tile sets; its
exact-path mask equals the 8x4 kernel's; other bin sizes and modes fall back unchanged."""
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


def _render(lr, s, k=3, carry=False, bin_size=32, owned=None, out=None, mask=False, shared=True):
    r = lr.Renderer(sorter_k=k, carry_colors=carry, bin_size=bin_size, shared_setup=shared)
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
        "dense_bins": scenegen.gaussian_particles(20_000, 96, 64, seed=11, sigma=0.05, size_px=(2.0, 6.0)),
        "big_near_quads": scenegen.frustum_parallelograms(300, 160, 96, seed=9, edge_range=(0.5, 6.0), far=8.0),
        "tiny": scenegen.frustum_parallelograms(40, 13, 7, seed=2, edge_range=(0.5, 3.0), far=10.0),
    }


@pytest.mark.parametrize("name", list(_scenes()))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_strip_matches_oracle(lr, name, k):
    s = _scenes()[name]
    out, st = _render(lr, s, k)
    assert st["status"] == 0
    _compare(out, st, oracle.render(s))


@pytest.mark.parametrize("name", ["particles", "layers_flat"])
def test_strip_carried_flat_colours(lr, name):
    s = _scenes()[name]
    out, st = _render(lr, s, 1, carry=True)
    _compare(out, st, oracle.render(s))


@pytest.mark.parametrize("name", ["layers", "particles"])
def test_strip_full_size(lr, name):
    s = {"layers": scenegen.config_layers_1080p, "particles": scenegen.config_particles_1080p}[name]()
    out, st = _render(lr, s, 1)
    assert st["status"] == 0
    _compare(out, st, oracle.render(s))


def test_strip_exact_mask_equals_half_blocks(lr):
    s = _scenes()["layers_vertex"]
    a, sa = _render(lr, s, 1, mask=True)
    b, sb = _render(lr, s, 1, mask=True, shared=False)
    assert sa["overflow_pixels"] == sb["overflow_pixels"] > 0
    assert torch.equal(a["exact_mask"], b["exact_mask"])
    assert torch.equal(a["count"], b["count"]) and torch.equal(a["hash"], b["hash"])


def test_strip_with_owned_tiles(lr):
    s = _scenes()["layers_vertex"]
    o = oracle.render(s)
    owner = PT.assign_tiles(s.width, s.height, 3)
    for rank in range(3):
        bits = torch.from_numpy(PT.owned_bitset(owner, rank).view(np.int32)).cuda()
        r = lr.Renderer(sorter_k=1, shared_setup=True)
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


@pytest.mark.parametrize("bin_size", [16, 64])
def test_strip_other_bin_sizes_fall_back(lr, bin_size):
    s = _scenes()["layers_vertex"]
    out, st = _render(lr, s, 1, bin_size=bin_size)
    _compare(out, st, oracle.render(s))


def test_strip_batch_of_views(lr):
    scenes = [scenegen.config_small_frustum(), scenegen.wavy_layers(200, 120, layers=8, nx=16, ny=8, seed=3),
              scenegen.gaussian_particles(5000, 128, 96, seed=2)]
    r = lr.Renderer(sorter_k=2, shared_setup=True, carry_colors=True)
    outs = r.render_batch([(lr.DeviceScene.from_scene(s), s.width, s.height) for s in scenes], count=True, hash=True)
    torch.cuda.synchronize()
    for s, o in zip(scenes, outs):
        ref = oracle.render(s)
        np.testing.assert_array_equal(o["count"].cpu().numpy().view(np.uint32), ref["count"])
        np.testing.assert_array_equal(o["hash"].cpu().numpy().view(np.uint64), ref["hash"])
        assert np.abs(o["rgba"].cpu().numpy().astype(np.float64) - ref["rgba"]).max() <= COLOR_TOL
    r.close()
