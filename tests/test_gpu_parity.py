"""Parity of the CUDA path with the CPU oracle (run on a GB300; marked gpu).

Bar: per-pixel fragment counts and coverage hashes bit-exact, setup records bit-exact,
linear fp32 RGBA within 1e-5 absolute per channel, 8-bit output within 1 LSB.
Every call goes through the C ABI (liblr.so) via the ctypes binding.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from scenegen import COLOR_FLAT, COLOR_VERTEX, Scene
from tests.scene_helpers import concat_scenes, rects_scene, tilted_plane_quad

pytestmark = pytest.mark.gpu

COLOR_TOL = 1e-5


@pytest.fixture(scope="module")
def lr():
    import paper_2405_13364_gb300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    P.load_library()
    return P


_renderers = {}


def renderer(lr, k=3):
    if k not in _renderers:
        _renderers[k] = lr.Renderer(sorter_k=k)
    return _renderers[k]


def gpu_render(lr, scene, k=3):
    r = renderer(lr, k)
    ds = lr.DeviceScene.from_scene(scene)
    out = r.render(ds, scene.width, scene.height, rgba8=True, count=True, hash=True)
    torch.cuda.synchronize()
    st = r.stats()
    res = dict(rgba=out["rgba"].cpu().numpy(), rgba8=out["rgba8"].cpu().numpy(),
               count=out["count"].cpu().numpy().view(np.uint32),
               hash=out["hash"].cpu().numpy().view(np.uint64), stats=st)
    return res


def assert_parity(g, o, tol=COLOR_TOL):
    np.testing.assert_array_equal(g["count"], o["count"])
    np.testing.assert_array_equal(g["hash"], o["hash"])
    d = np.abs(g["rgba"].astype(np.float64) - o["rgba"].astype(np.float64))
    assert d.max() <= tol, f"max colour error {d.max()} at {np.unravel_index(d.argmax(), d.shape)}"
    d8 = np.abs(g["rgba8"].astype(np.int32) - o["rgba8"].astype(np.int32))
    assert d8.max() <= 1
    assert g["stats"]["fragments"] == int(o["count"].sum())


def small_scenes():
    return {
        "frustum256": scenegen.config_small_frustum(),
        "frustum_ragged": scenegen.frustum_parallelograms(3000, 200, 141, seed=4),
        "layers_vertex": scenegen.wavy_layers(333, 190, layers=32, nx=48, ny=24, seed=1),
        "layers_flat": scenegen.wavy_layers(256, 256, layers=24, nx=32, ny=32, seed=2,
                                            color_mode=COLOR_FLAT),
        "particles": scenegen.gaussian_particles(60_000, 320, 180, seed=3),
        "big_near_quads": scenegen.frustum_parallelograms(300, 160, 96, seed=9,
                                                          edge_range=(0.5, 6.0), far=8.0),
    }


@pytest.mark.parametrize("name", list(small_scenes()))
@pytest.mark.parametrize("k", [1, 3, 8])
def test_render_matches_oracle(lr, name, k):
    s = small_scenes()[name]
    o = oracle.render(s)
    g = gpu_render(lr, s, k)
    assert g["stats"]["status"] == 0
    assert_parity(g, o)
    if k == 1 and name.startswith("layers"):
        # interpenetrating layers: the 1-slot sorter cannot order them; the exact
        # overflow path must have run
        assert g["stats"]["overflow_pixels"] > 0


def test_setup_records_bit_exact(lr):
    s = scenegen.frustum_parallelograms(5000, 300, 200, seed=5, edge_range=(0.05, 5.0), far=30.0)
    r = renderer(lr)
    ds = lr.DeviceScene.from_scene(s)
    out = r.make_outputs(s.width, s.height)
    view = r.view_struct(ds, s.width, s.height, out)
    r.render_views([view])
    torch.cuda.synchronize()
    from paper_2405_13364_gb300 import _binding as B
    lay = B.lr_workspace_layout(r.ctx, [view], r._ws_bytes)
    base = (int(r._ws.data_ptr()) + 255) & ~255
    off = base - int(r._ws.data_ptr())
    ws = r._ws
    q = s.num_quads

    def grab(o, nbytes, dtype):
        return ws[off + o: off + o + nbytes].cpu().numpy().view(dtype)

    rec = grab(lay.rec, 64 * q, np.int32).reshape(q, 16)
    xy = rec[:, 0:8]
    qq = rec[:, 8:12].view(np.float32)
    rect = grab(lay.rec_rect, 8 * q, np.uint32).reshape(q, 2)
    info = grab(lay.rec_info, 4 * q, np.uint32)
    os_ = oracle.setup(s)
    np.testing.assert_array_equal(info >> 8, os_["status"].astype(np.uint32))
    vis = os_["status"] == 0
    assert vis.sum() > 1000
    np.testing.assert_array_equal(xy[vis][:, 0::2], os_["X"][vis])
    np.testing.assert_array_equal(xy[vis][:, 1::2], os_["Y"][vis])
    np.testing.assert_array_equal(qq[vis].view(np.uint32), os_["q"][vis].view(np.uint32))
    bb = os_["bbox"][vis]
    np.testing.assert_array_equal(rect[vis][:, 0] & 0xFFFF, bb[:, 0])
    np.testing.assert_array_equal(rect[vis][:, 0] >> 16, bb[:, 1])
    np.testing.assert_array_equal(rect[vis][:, 1] & 0xFFFF, bb[:, 2])
    np.testing.assert_array_equal(rect[vis][:, 1] >> 16, bb[:, 3])
    st = r.stats()
    assert st["quads_visible"] == int(vis.sum())
    for reason in range(1, 7):
        assert st["culled"][reason] == int((os_["status"] == reason).sum())


def test_closed_form_rects(lr):
    c = np.array([[0.9, 0.1, 0.2, 0.6], [0.1, 0.8, 0.3, 0.7]], np.float32)
    s = rects_scene([(2.0, 2.0, 10.0, 10.0), (6.0, 6.0, 14.0, 14.0)], depths=[1.0, 2.0], colors=c)
    g = gpu_render(lr, s)
    assert_parity(g, oracle.render(s))
    assert np.all(g["count"][6:10, 6:10] == 2)


def test_equal_depth_ties(lr):
    rng = np.random.default_rng(0)
    rects = [(1.0, 1.0, 15.0, 15.0)] * 40
    cols = np.concatenate([rng.random((40, 3)), rng.uniform(0.1, 0.5, (40, 1))], 1)
    s = rects_scene(rects, colors=cols)
    for k in (1, 3):
        assert_parity(gpu_render(lr, s, k), oracle.render(s))


def test_interpenetrating_planes(lr):
    a = tilted_plane_quad(96, 64, depth=3.0, slope_x=0.9, slope_y=0.2, half=1.5)
    b = tilted_plane_quad(96, 64, depth=3.0, slope_x=-0.9, slope_y=-0.1, half=1.5,
                          flat_color=(0.1, 0.2, 0.9, 0.4))
    s = concat_scenes(a, b)
    for k in (1, 2, 3):
        assert_parity(gpu_render(lr, s, k), oracle.render(s))


def test_high_density_bin_global_sort(lr):
    # ~20k tiny particles inside a few bins: more than 4096 references per bin
    s = scenegen.gaussian_particles(20_000, 96, 64, seed=11, sigma=0.05, size_px=(2.0, 6.0))
    g = gpu_render(lr, s)
    assert g["stats"]["bins_high"] > 0
    assert_parity(g, oracle.render(s))


def test_empty_and_all_culled(lr):
    m, n, f = scenegen.perspective(64, 48)
    pos = np.zeros((4, 3), np.float32)
    pos[:, 2] = 5.0   # behind the camera
    s = Scene(pos, None, np.ones((1, 4), np.float32), COLOR_FLAT, m, float(n), float(f), 64, 48)
    g = gpu_render(lr, s)
    assert np.all(g["rgba"] == 0) and np.all(g["count"] == 0)
    s0 = Scene(np.zeros((0, 3), np.float32), None, np.zeros((0, 4), np.float32), COLOR_FLAT, m,
               float(n), float(f), 64, 48)
    g0 = gpu_render(lr, s0)
    assert np.all(g0["rgba"] == 0)


def test_bad_index_reported(lr):
    s = scenegen.wavy_layers(64, 64, layers=2, nx=4, ny=4, seed=1)
    idx = s.indices.copy()
    idx[3, 2] = s.num_vertices + 7
    bad = Scene(s.positions, idx, s.colors, s.color_mode, s.view_proj, s.near, s.far, 64, 64)
    r = renderer(lr)
    ds = lr.DeviceScene.from_scene(bad)
    with pytest.raises(lr.LrError) as e:
        r.render(ds, 64, 64)
    assert e.value.status == -1
    torch.cuda.synchronize()


def test_small_workspace_overflow_then_retry(lr):
    from paper_2405_13364_gb300 import _binding as B
    s = scenegen.frustum_parallelograms(400, 256, 256, seed=3, edge_range=(1.0, 8.0), far=10.0)
    r = lr.Renderer(sorter_k=3, ref_factor=1)
    ds = lr.DeviceScene.from_scene(s)
    out = r.make_outputs(256, 256, count=True)
    view = r.view_struct(ds, 256, 256, out)
    need = B.lr_workspace_size_batch(r.ctx, [view])
    ptr, nbytes = r.workspace(need)
    B.lr_render_batch(r.ctx, [view], ptr, nbytes, torch.cuda.current_stream().cuda_stream)
    st = B.lr_get_stats(r.ctx, raise_on_error=False)
    if st.bin_refs > st.bin_refs_capacity:
        assert st.status == B.LR_ERR_OVERFLOW
    # the Renderer grows the workspace and succeeds
    o = r.render(ds, 256, 256, count=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(o["count"].cpu().numpy().view(np.uint32), oracle.render(s)["count"])
    r.close()


def test_batch_equals_single(lr):
    scenes = [scenegen.config_small_frustum(),
              scenegen.wavy_layers(200, 120, layers=8, nx=16, ny=8, seed=3),
              scenegen.gaussian_particles(5000, 128, 96, seed=2)]
    r = renderer(lr)
    items = [(lr.DeviceScene.from_scene(s), s.width, s.height) for s in scenes]
    outs = r.render_batch(items, count=True, hash=True)
    torch.cuda.synchronize()
    for s, o in zip(scenes, outs):
        single = gpu_render(lr, s)
        np.testing.assert_array_equal(o["rgba"].cpu().numpy(), single["rgba"])
        np.testing.assert_array_equal(o["count"].cpu().numpy().view(np.uint32), single["count"])
        np.testing.assert_array_equal(o["hash"].cpu().numpy().view(np.uint64), single["hash"])


def test_deterministic(lr):
    s = scenegen.gaussian_particles(30_000, 256, 160, seed=8)
    a = gpu_render(lr, s)
    b = gpu_render(lr, s)
    np.testing.assert_array_equal(a["rgba"], b["rgba"])
    np.testing.assert_array_equal(a["hash"], b["hash"])


@pytest.mark.parametrize("name", ["frustum256", "layers_flat", "particles"])
@pytest.mark.parametrize("k", [1, 3])
def test_carried_flat_colours_bitwise(lr, name, k):
    # a flat-colour scene through the colour-carrying rasteriser (each triangle's colour with
    # zero increments and the scale 1) and through the one that gathers colours at blend
    # time: the same fragments composited in the same order with the same arithmetic, so
    # the two images are equal bit for bit
    s = small_scenes()[name]
    assert s.color_mode == COLOR_FLAT
    imgs = []
    for carry in (False, True):
        r = lr.Renderer(sorter_k=k, carry_colors=carry)
        out = r.render(lr.DeviceScene.from_scene(s), s.width, s.height, rgba8=True)
        torch.cuda.synchronize()
        assert r.stats()["status"] == 0
        imgs.append((out["rgba"].cpu().numpy().view(np.uint32), out["rgba8"].cpu().numpy()))
        r.close()
    np.testing.assert_array_equal(imgs[0][0], imgs[1][0])
    np.testing.assert_array_equal(imgs[0][1], imgs[1][1])
