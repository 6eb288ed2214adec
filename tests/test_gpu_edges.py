"""Edge cases of the CUDA path against the oracle: tiny and maximum resolutions, ragged
sizes, screen-filling and guard-band quads, shared edges through pixel centres, equal
depths in dense stacks, degenerate triangles, every sorter capacity, mixed colour modes in
one batch."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from scenegen import COLOR_FLAT, COLOR_VERTEX, Scene
from tests.scene_helpers import rects_scene, screen_quads_scene, shared_grid
from tests.test_gpu_parity import assert_parity, gpu_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import paper_2405_13364_gb300 as P
    P.load_library()
    return P


@pytest.mark.parametrize("wh", [(1, 1), (1, 37), (37, 1), (33, 31), (65, 97)])
def test_tiny_and_ragged_sizes(lr, wh):
    w, h = wh
    s = scenegen.frustum_parallelograms(400, w, h, seed=w * 100 + h, edge_range=(0.3, 3.0), far=10.0)
    assert_parity(gpu_render(lr, s), oracle.render(s))


def test_max_resolution(lr):
    s = scenegen.frustum_parallelograms(20_000, 2560, 2048, seed=5, edge_range=(0.05, 2.0), far=30.0)
    assert_parity(gpu_render(lr, s), oracle.render(s))


def test_screen_filling_and_guard_band_quads(lr):
    m, n, f = scenegen.perspective(320, 200)
    rng = np.random.default_rng(4)
    pos = []
    # quads much larger than the screen (still inside the guard band) at several depths
    for d in (1.0, 1.5, 2.5, 4.0):
        e = 1.6 * d
        pos += [(-e, -e, -d), (e, -e * 0.9, -d - 0.3), (e * 1.1, e, -d), (-e, e * 1.2, -d + 0.2)]
    # quads crossing the guard band (culled) and the near plane (culled)
    pos += [(-0.5, -0.5, -2), (9000.0, -0.5, -2), (0.5, 0.5, -2), (-0.5, 0.5, -2)]
    pos += [(-0.5, -0.5, -2), (0.5, -0.5, -0.01), (0.5, 0.5, -2), (-0.5, 0.5, -2)]
    q = len(pos) // 4
    col = np.concatenate([rng.random((q, 3)), rng.uniform(0.2, 0.7, (q, 1))], 1).astype(np.float32)
    s = Scene(np.array(pos, np.float32), None, col, COLOR_FLAT, m, float(n), float(f), 320, 200)
    for k in (1, 3):
        g = gpu_render(lr, s, k)
        assert_parity(g, oracle.render(s))
    assert g["stats"]["culled"][4] == 1 and g["stats"]["culled"][3] == 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_edges_through_pixel_centres(lr, seed):
    vxy, idx = shared_grid(12, 9, -3.0, -2.0, 67.0, 50.0, jitter=0.35, seed=seed, exact_centres=True)
    rng = np.random.default_rng(seed)
    cols = np.concatenate([rng.random((idx.shape[0], 3)), rng.uniform(0.2, 0.8, (idx.shape[0], 1))], 1)
    s = screen_quads_scene(vxy, 64, 48, cols, indices=idx)
    g = gpu_render(lr, s)
    assert g["count"].min() == 1 and g["count"].max() == 1
    assert_parity(g, oracle.render(s))


def test_dense_equal_depth_stack(lr):
    # 9000 identical-depth rectangles over a small region: high-density bins, every key ties
    rng = np.random.default_rng(3)
    rects = []
    for _ in range(9000):
        x0, y0 = rng.uniform(0, 40, 2)
        rects.append((float(np.floor(x0 * 4) / 4), float(np.floor(y0 * 4) / 4),
                      float(np.floor(x0 * 4) / 4 + 8.0), float(np.floor(y0 * 4) / 4 + 6.0)))
    cols = np.concatenate([rng.random((9000, 3)), rng.uniform(0.02, 0.2, (9000, 1))], 1)
    s = rects_scene(rects, width=64, height=64, colors=cols)
    for k in (1, 3):
        g = gpu_render(lr, s, k)
        assert g["stats"]["bins_high"] > 0
        assert_parity(g, oracle.render(s))


def test_degenerate_triangles(lr):
    # quads with one zero-area triangle (three collinear vertices) next to normal ones
    xy = []
    cols = []
    rng = np.random.default_rng(8)
    for i in range(40):
        x, y = rng.uniform(2, 60, 2)
        if i % 2:
            xy += [(x, y), (x + 6, y), (x + 12, y), (x + 3, y + 7)]      # T0 degenerate
        else:
            xy += [(x, y), (x + 6, y + 1), (x + 6, y + 1), (x, y + 7)]   # repeated vertex
        cols.append([*rng.random(3), 0.5])
    s = screen_quads_scene(np.array(xy), 64, 64, np.array(cols))
    assert_parity(gpu_render(lr, s), oracle.render(s))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8, 12])
def test_every_sorter_capacity(lr, k):
    s = scenegen.wavy_layers(160, 96, layers=20, nx=20, ny=10, seed=6, dz=0.25)
    assert_parity(gpu_render(lr, s, k), oracle.render(s))


def test_mixed_colour_modes_in_one_batch(lr):
    scenes = [scenegen.wavy_layers(128, 96, layers=10, nx=12, ny=8, seed=1, color_mode=COLOR_VERTEX),
              scenegen.frustum_parallelograms(2000, 128, 96, seed=2),
              scenegen.gaussian_particles(10_000, 128, 96, seed=3)]
    r = lr.Renderer(sorter_k=3)
    items = [(lr.DeviceScene.from_scene(s), s.width, s.height) for s in scenes]
    outs = r.render_batch(items, count=True, hash=True, rgba8=True)
    torch.cuda.synchronize()
    for s, o in zip(scenes, outs):
        g = dict(rgba=o["rgba"].cpu().numpy(), rgba8=o["rgba8"].cpu().numpy(),
                 count=o["count"].cpu().numpy().view(np.uint32),
                 hash=o["hash"].cpu().numpy().view(np.uint64),
                 stats=dict(fragments=int(o["count"].cpu().numpy().astype(np.int64).sum())))
        assert_parity(g, oracle.render(s))
    r.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_concave_and_crossed_quads(lr, seed):
    # four random vertices per quad within a few pixels: convex, concave and self-crossing
    # (bow-tie) quads, so the two triangles come with every combination of orientations (the
    # rasteriser derives one triangle's diagonal coverage from the other's), vertices on
    # pixel centres half of the time
    rng = np.random.default_rng(seed)
    xy = []
    for i in range(600):
        c = rng.uniform(4, 92, 2)
        v = c + rng.uniform(-7, 7, (4, 2))
        if i % 2:
            v = np.floor(v) + 0.5
        xy += [tuple(p) for p in v]
    cols = np.concatenate([rng.random((600, 3)), rng.uniform(0.1, 0.6, (600, 1))], 1)
    s = screen_quads_scene(np.array(xy), 96, 96, cols)
    o = oracle.render(s)
    for k in (1, 3):
        g = gpu_render(lr, s, k)
        assert_parity(g, o)
