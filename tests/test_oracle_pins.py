"""Pins for the CPU oracle: checks against facts fixed by geometry and algebra, not by
re-running the oracle's own formulas.

* closed-form coverage of rectangles (fill rule + snapping), golden cases in
  tests/golden/closed_form_rects.txt
* closed-form composites of one and two layers, depth order independent of submission
  order, equal-depth ties resolved by quad index
* exactly-once coverage of shared edges and vertices (tilings)
* invariance of the image to the order of the input quads
* brute force on 16x16 images (a second enumeration, Python integers)
* the depth key equals 1/w interpolated linearly in screen space (fp64 plane fit)
* perspective-correct vertex colours equal an fp64 rational fit
* the fp32 composite is within 1e-6 of the fp64 composite of the same order
* the fp64 gradient equals central finite differences (exact up to rounding, since the
  composite is affine in every single colour channel and the loss is quadratic)
* 8-bit conversion values and the cull rules
"""
import os

import numpy as np
import pytest

import oracle
import scenegen
from oracle import brute
from scenegen import COLOR_FLAT, COLOR_VERTEX, Scene
from tests.scene_helpers import (concat_scenes, permute_scene, rects_scene, screen_quads_scene,
                                 shared_grid, tilted_plane_quad)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_rects.txt")


def _golden_rects():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = line.split()
        rows.append(tuple(float(x) for x in v[:4]) + tuple(int(x) for x in v[4:]))
    return rows


@pytest.mark.parametrize("reverse", [False, True])
@pytest.mark.parametrize("rotate", [0, 1])
def test_rect_coverage_closed_form(reverse, rotate):
    for x0, y0, x1, y1, pxa, pxb, pya, pyb in _golden_rects():
        s = rects_scene([(x0, y0, x1, y1)], reverse=reverse, rotate=rotate)
        r = oracle.render(s)
        want = np.zeros((16, 16), np.uint32)
        if pxa <= pxb and pya <= pyb:
            want[pya:pyb + 1, pxa:pxb + 1] = 1
        np.testing.assert_array_equal(r["count"], want, err_msg=str((x0, y0, x1, y1)))
        # one layer over black: colour = a*c, alpha = a (fp32 products)
        a = np.float32(0.5)
        c = np.array([0.2, 0.4, 0.6], np.float32)
        cov = want.astype(bool)
        np.testing.assert_array_equal(r["rgba"][cov][:, :3], np.broadcast_to(a * c, (cov.sum(), 3)))
        np.testing.assert_array_equal(r["rgba"][cov][:, 3], np.full(cov.sum(), a))
        assert np.all(r["rgba"][~cov] == 0)


def test_snap_rounds_half_to_even():
    # x0 = 2.5 + 1/512 lies exactly halfway between two subpixel positions: 640.5 -> 640
    # (even), i.e. x0 snaps to 2.5 and the centre 2.5 of column 2 is on an owned edge.
    s = rects_scene([(2.5 + 1 / 512, 0.5, 6.5, 1.5)])
    st = oracle.setup(s)
    assert st["X"][0, 0] == 640
    assert oracle.render(s)["count"][0, 2] == 1
    # 3.5 + 1/512 -> 896.5 -> 896 (even) again; 2.5 + 3/512 -> 641.5 -> 642 (even)
    s2 = rects_scene([(2.5 + 3 / 512, 0.5, 3.5 + 1 / 512, 1.5)])
    st2 = oracle.setup(s2)
    assert st2["X"][0, 0] == 642 and st2["X"][0, 1] == 896
    assert oracle.render(s2)["count"][0, 2] == 0   # centre 2.5 < 642/256


def test_two_layers_closed_form_and_order():
    near_rect, far_rect = (2.0, 2.0, 10.0, 10.0), (6.0, 6.0, 14.0, 14.0)
    cn = np.array([0.9, 0.1, 0.2, 0.6], np.float32)
    cf = np.array([0.1, 0.8, 0.3, 0.7], np.float32)
    out = []
    for order in ((0, 1), (1, 0)):
        rects = [near_rect, far_rect]
        depths = [1.0, 2.0]
        cols = [cn, cf]
        s = rects_scene([rects[i] for i in order], depths=[depths[i] for i in order],
                        colors=np.stack([cols[i] for i in order]))
        out.append(oracle.render(s))
    np.testing.assert_array_equal(out[0]["rgba"], out[1]["rgba"])
    r = out[0]
    an, af = float(cn[3]), float(cf[3])
    want_overlap = an * cn[:3].astype(np.float64) + (1 - an) * af * cf[:3].astype(np.float64)
    want_alpha = an + (1 - an) * af
    got = r["rgba"][6:10, 6:10].reshape(-1, 4).astype(np.float64)
    assert np.abs(got[:, :3] - want_overlap).max() < 1e-6
    assert np.abs(got[:, 3] - want_alpha).max() < 1e-6
    assert np.all(r["count"][6:10, 6:10] == 2)
    # near only / far only
    assert np.abs(r["rgba"][3, 3, :3] - an * cn[:3]).max() < 1e-7
    assert np.abs(r["rgba"][12, 12, :3] - af * cf[:3]).max() < 1e-7


def test_equal_depth_tie_higher_index_on_top():
    c0 = np.array([1.0, 0.0, 0.0, 0.5], np.float32)
    c1 = np.array([0.0, 0.0, 1.0, 0.5], np.float32)
    s = rects_scene([(2, 2, 10, 10), (2, 2, 10, 10)], colors=np.stack([c0, c1]))
    px = oracle.render(s)["rgba"][5, 5].astype(np.float64)
    # quad 1 (higher index) is composited last, i.e. in front
    want = 0.5 * c1[:3] + 0.5 * 0.5 * c0[:3]
    assert np.abs(px[:3] - want).max() < 1e-7
    fr = oracle.pixel_fragments(s, 5, 5)
    assert list(fr["quad"]) == [0, 1]


def test_exactly_once_jittered_grid():
    # a jittered grid covering the screen with margin: every pixel exactly once
    vxy, idx = shared_grid(9, 7, -3.0, -2.0, 35.0, 26.0, jitter=0.3, seed=3)
    cols = np.tile([[0.5, 0.5, 0.5, 0.5]], (idx.shape[0], 1))
    s = screen_quads_scene(vxy, 32, 24, cols, indices=idx)
    r = oracle.render(s)
    assert r["count"].min() == 1 and r["count"].max() == 1


@pytest.mark.parametrize("seed", [0, 1])
def test_exactly_once_edges_through_centres(seed):
    # vertices on pixel centres: shared edges and vertices lie exactly on sample points
    vxy, idx = shared_grid(8, 8, -2.0, -2.0, 34.0, 34.0, jitter=0.35, seed=seed,
                           exact_centres=True)
    cols = np.tile([[0.5, 0.5, 0.5, 0.5]], (idx.shape[0], 1))
    s = screen_quads_scene(vxy, 32, 32, cols, indices=idx)
    r = oracle.render(s)
    assert r["count"].max() == 1
    assert r["count"].min() == 1


def test_exactly_once_under_perspective():
    # the 1080p layer generator's grids: within one layer no pixel is covered twice
    s = scenegen.wavy_layers(64, 48, layers=1, nx=24, ny=12, seed=5, color_mode=COLOR_FLAT,
                             half_h=1.0, d0=1.5, amplitude=0.05)
    r = oracle.render(s)
    assert r["count"].max() == 1
    # the projected layer covers the screen centre region completely
    assert np.all(r["count"][12:36, 16:48] == 1)


@pytest.mark.parametrize("make", ["frustum", "layers"])
def test_permutation_invariance(make):
    if make == "frustum":
        s = scenegen.frustum_parallelograms(600, 64, 64, seed=7)
    else:
        s = scenegen.wavy_layers(64, 64, layers=6, nx=8, ny=8, seed=2, color_mode=COLOR_FLAT)
    r0 = oracle.render(s)
    assert r0["stats"]["key_ties"] == 0
    perm = np.random.default_rng(11).permutation(s.num_quads)
    r1 = oracle.render(permute_scene(s, perm))
    np.testing.assert_array_equal(r0["rgba"], r1["rgba"])
    np.testing.assert_array_equal(r0["count"], r1["count"])


def _tiny_scenes():
    out = []
    for seed in range(6):
        s = scenegen.frustum_parallelograms(24, 16, 16, seed=seed, edge_range=(0.5, 4.0), far=12.0)
        out.append(s)
    # near-plane crossers and guard-band quads
    m, n, f = scenegen.perspective(16, 16)
    rng = np.random.default_rng(9)
    pos = []
    for _ in range(12):
        c = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), -rng.uniform(0.05, 3.0)])
        e1, e2 = rng.normal(size=3) * 1.2, rng.normal(size=3) * 1.2
        pos += [c - e1 / 2 - e2 / 2, c + e1 / 2 - e2 / 2, c + e1 / 2 + e2 / 2, c - e1 / 2 + e2 / 2]
    col = np.concatenate([rng.random((12, 3)), rng.uniform(0.2, 0.8, (12, 1))], 1)
    out.append(Scene(np.array(pos, np.float32), None, col.astype(np.float32), COLOR_FLAT, m,
                     float(n), float(f), 16, 16))
    # per-vertex colours, shared vertices, interpenetrating layers
    out.append(scenegen.wavy_layers(16, 16, layers=4, nx=3, ny=3, seed=1, half_h=1.5,
                                    amplitude=0.3, dz=0.2))
    # ragged 13x11 image
    out.append(scenegen.frustum_parallelograms(20, 13, 11, seed=42, edge_range=(0.5, 3.0), far=10.0))
    return out


@pytest.mark.parametrize("k", range(9))
def test_brute_force_tiny(k):
    s = _tiny_scenes()[k]
    r = oracle.render(s)
    rgba, count, hsh = brute.render(s)
    np.testing.assert_array_equal(r["count"], count)
    np.testing.assert_array_equal(r["hash"], hsh)
    np.testing.assert_array_equal(r["rgba"], rgba)
    assert r["count"].sum() > 0


@pytest.mark.parametrize("k", [0, 6, 7, 8])
def test_render_pixels_equals_brute_force(k):
    # the per-pixel entry point (its own gather / sort / composite loop) on every pixel of a
    # tiny scene, in a shuffled order, against the independent brute force
    s = _tiny_scenes()[k]
    rgba, count, hsh = brute.render(s)
    ys, xs = np.meshgrid(np.arange(s.height), np.arange(s.width), indexing="ij")
    perm = np.random.default_rng(k).permutation(xs.size)
    xs, ys = xs.reshape(-1)[perm], ys.reshape(-1)[perm]
    p = oracle.render_pixels(s, xs, ys)
    np.testing.assert_array_equal(p["count"], count[ys, xs])
    np.testing.assert_array_equal(p["hash"], hsh[ys, xs])
    np.testing.assert_array_equal(p["rgba"], rgba[ys, xs])


def test_render_pixels_equals_full_render_on_dense_scenes():
    # sampled pixels of dense scenes (deep interpenetrating layers, particles), including the
    # image corners and out-of-order repeats, bit for bit against the full-image render
    for s in (scenegen.wavy_layers(200, 120, layers=32, nx=40, ny=20, seed=5),
              scenegen.gaussian_particles(20_000, 160, 90, seed=6)):
        full = oracle.render(s)
        rng = np.random.default_rng(1)
        xs = np.concatenate([rng.integers(0, s.width, 500), [0, s.width - 1, 0, s.width - 1, 7, 7]])
        ys = np.concatenate([rng.integers(0, s.height, 500), [0, 0, s.height - 1, s.height - 1, 3, 3]])
        p = oracle.render_pixels(s, xs, ys)
        np.testing.assert_array_equal(p["count"], full["count"][ys, xs])
        np.testing.assert_array_equal(p["hash"], full["hash"][ys, xs])
        np.testing.assert_array_equal(p["rgba"], full["rgba"][ys, xs])
        assert p["count"].max() > 20


def test_depth_key_is_screen_linear_inverse_w():
    s = tilted_plane_quad(64, 64, depth=3.0, slope_x=0.8, slope_y=-0.5, half=1.2)
    st = oracle.setup(s)
    assert st["status"][0] == 0
    X = st["X"][0].astype(np.float64) / 256.0
    Y = st["Y"][0].astype(np.float64) / 256.0
    q = st["q"][0].astype(np.float64)
    checked = 0
    for t, (a, b, c) in enumerate(((0, 1, 2), (0, 2, 3))):
        A = np.array([[X[a], Y[a], 1.0], [X[b], Y[b], 1.0], [X[c], Y[c], 1.0]])
        coef = np.linalg.solve(A, q[[a, b, c]])
        for py in range(0, 64, 3):
            for px in range(0, 64, 3):
                fr = oracle.pixel_fragments(s, px, py)
                for key, tri in zip(fr["key"], fr["tri"]):
                    if tri != t:
                        continue
                    want = coef @ np.array([px + 0.5, py + 0.5, 1.0])
                    assert abs(float(key) - want) <= 4e-7 * abs(want)
                    checked += 1
    assert checked > 50


def test_interpenetrating_planes_order():
    a = tilted_plane_quad(48, 48, depth=3.0, slope_x=0.9, slope_y=0.0, half=1.5,
                          flat_color=(1.0, 0.0, 0.0, 0.5))
    b = tilted_plane_quad(48, 48, depth=3.0, slope_x=-0.9, slope_y=0.0, half=1.5,
                          flat_color=(0.0, 0.0, 1.0, 0.5))
    s = concat_scenes(a, b)
    r = oracle.render(s)
    img = r["rgba"].astype(np.float64)
    # plane a: depth 3 + 0.9x, plane b: 3 - 0.9x. Along the ray through screen column px
    # (view-space slope u < 0 left of centre) a is nearer iff u < 0.
    near_a = 0.5 * np.array([1, 0, 0]) + 0.25 * np.array([0, 0, 1])
    near_b = 0.5 * np.array([0, 0, 1]) + 0.25 * np.array([1, 0, 0])
    both = np.argwhere(r["count"] == 2)
    assert len(both) > 100
    n_left = n_right = 0
    for py, px in both:
        u = (2.0 * (px + 0.5) / 48 - 1.0)
        if abs(u) < 0.05:
            continue
        want = near_a if u < 0 else near_b
        assert np.abs(img[py, px, :3] - want).max() < 1e-6, (px, py)
        n_left += u < 0
        n_right += u > 0
    assert n_left > 20 and n_right > 20


def test_perspective_correct_vertex_colour():
    vc = np.array([[1.0, 0.0, 0.0, 0.2], [0.0, 1.0, 0.0, 0.4], [0.0, 0.0, 1.0, 0.6],
                   [1.0, 1.0, 0.0, 0.8]], np.float32)
    s = tilted_plane_quad(64, 64, depth=2.0, slope_x=1.5, slope_y=0.3, half=1.0,
                          color_mode=COLOR_VERTEX, vertex_colors=vc)
    st = oracle.setup(s)
    X = st["X"][0].astype(np.float64) / 256.0
    Y = st["Y"][0].astype(np.float64) / 256.0
    q = st["q"][0].astype(np.float64)
    checked = 0
    for t, (a, b, c) in enumerate(((0, 1, 2), (0, 2, 3))):
        A = np.array([[X[a], Y[a], 1.0], [X[b], Y[b], 1.0], [X[c], Y[c], 1.0]])
        den = np.linalg.solve(A, q[[a, b, c]])
        num = np.linalg.solve(A, q[[a, b, c], None] * vc[[a, b, c]].astype(np.float64))
        for py in range(0, 64, 4):
            for px in range(0, 64, 4):
                fr = oracle.pixel_fragments(s, px, py)
                for rgba, tri in zip(fr["rgba"], fr["tri"]):
                    if tri != t:
                        continue
                    p = np.array([px + 0.5, py + 0.5, 1.0])
                    want = (p @ num) / (p @ den)
                    assert np.abs(rgba - want).max() < 2e-6
                    checked += 1
    assert checked > 20


def test_fp32_composite_close_to_fp64():
    r = oracle.render(scenegen.frustum_parallelograms(2000, 128, 128, seed=0), want64=True)
    assert np.abs(r["rgba"] - r["rgba64"]).max() < 1e-6
    # deep stack: 300 layers of alpha 0.3 on one pixel region
    rects = [(1.0, 1.0, 7.0, 7.0)] * 300
    rng = np.random.default_rng(0)
    cols = np.concatenate([rng.random((300, 3)), rng.uniform(0.02, 0.3, (300, 1))], 1)
    s = rects_scene(rects, colors=cols, depths=list(np.linspace(1.0, 3.0, 300)))
    r = oracle.render(s, want64=True)
    assert r["count"].max() == 300
    assert np.abs(r["rgba"] - r["rgba64"]).max() < 1e-5


def _small_diff_scene():
    return scenegen.wavy_layers(48, 40, layers=6, nx=10, ny=8, seed=3, color_mode=COLOR_FLAT,
                                half_h=1.3, dz=0.4)


def test_backward_matches_central_differences():
    s = _small_diff_scene()
    target = oracle.render(s.with_colors(scenegen.perturbed_target_colors(s.colors, seed=1)))["rgba"]
    col64 = s.colors.astype(np.float64)
    img = oracle.render64(s, col64)
    g = oracle.backward(s, oracle.loss_l2_grad(img, target), col64)
    rng = np.random.default_rng(2)
    visible = np.nonzero(np.abs(g).sum(1) > 0)[0]
    picks = rng.choice(visible, 16, replace=False)
    h = 1e-3
    for j in picks:
        for ch in range(4):
            cp, cm = col64.copy(), col64.copy()
            cp[j, ch] += h
            cm[j, ch] -= h
            lp = oracle.loss_l2(oracle.render64(s, cp), target)
            lm = oracle.loss_l2(oracle.render64(s, cm), target)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[j, ch]) <= 1e-9 + 1e-7 * abs(g[j, ch]), (j, ch, fd, g[j, ch])


def test_backward_one_layer_closed_form():
    c = np.array([[0.3, 0.6, 0.9, 0.4]], np.float32)
    s = rects_scene([(2.0, 2.0, 6.0, 5.0)], colors=c)      # 4 x 3 = 12 pixels
    target = np.zeros((16, 16, 4), np.float32)
    img = oracle.render64(s)
    g = oracle.backward(s, oracle.loss_l2_grad(img, target))
    a, col = 0.4, c[0, :3].astype(np.float64)
    # C = a c: dL/dc = sum 2 C a, dL/da = sum_ch 2 C_ch c_ch, over 12 pixels
    want_c = 12 * 2 * (a * col) * a
    want_a = 12 * np.sum(2 * (a * col) * col)
    assert np.abs(g[0, :3] - want_c).max() < 1e-6
    assert abs(g[0, 3] - want_a) < 1e-6


def test_u8_conversion_values():
    cols = np.array([[0.5, 0.25, 1.0, 1.0], [2.0, -1.0, 0.0, 1.0]], np.float32)
    s = rects_scene([(0, 0, 4, 4), (8, 8, 12, 12)], colors=cols)
    r = oracle.render(s)
    # 0.5*255 = 127.5 -> 128 (half to even), 0.25*255 = 63.75 -> 64, 1 -> 255
    assert list(r["rgba8"][1, 1]) == [128, 64, 255, 255]
    # clamped: 2 -> 255, -1 -> 0
    assert list(r["rgba8"][9, 9]) == [255, 0, 0, 255]
    assert list(r["rgba8"][5, 5]) == [0, 0, 0, 0]


def test_cull_rules():
    m, n, f = scenegen.perspective(32, 32)
    quads = {
        "visible": [(-0.5, -0.5, -2), (0.5, -0.5, -2), (0.5, 0.5, -2), (-0.5, 0.5, -2)],
        "depth": [(-0.5, -0.5, -2), (0.5, -0.5, -2), (0.5, 0.5, -0.05), (-0.5, 0.5, -2)],
        "guard": [(-0.5, -0.5, -2), (3000.0, -0.5, -2), (0.5, 0.5, -2), (-0.5, 0.5, -2)],
        "nonfinite": [(-0.5, -0.5, -2), (np.nan, -0.5, -2), (0.5, 0.5, -2), (-0.5, 0.5, -2)],
        "degenerate": [(0.0, 0.0, -2), (0.1, 0.1, -2), (0.2, 0.2, -2), (0.3, 0.3, -2)],
        "no_pixel": [(0.001, 0.001, -2), (0.002, 0.001, -2), (0.002, 0.002, -2), (0.001, 0.002, -2)],
        "far": [(-0.5, -0.5, -200), (0.5, -0.5, -200), (0.5, 0.5, -200), (-0.5, 0.5, -200)],
    }
    names = list(quads)
    pos = np.array([p for k in names for p in quads[k]], np.float32)
    col = np.tile([[0.5, 0.5, 0.5, 0.5]], (len(names), 1)).astype(np.float32)
    s = Scene(pos, None, col, COLOR_FLAT, m, float(n), float(f), 32, 32)
    st = oracle.setup(s)["status"]
    want = {"visible": 0, "depth": 3, "guard": 4, "nonfinite": 2, "degenerate": 5,
            "no_pixel": 6, "far": 3}
    assert [int(x) for x in st] == [want[k] for k in names]
    # bad index
    s2 = Scene(pos[:4], np.array([[0, 1, 2, 7]], np.uint32), col[:1], COLOR_FLAT, m, float(n),
               float(f), 32, 32)
    assert oracle.setup(s2)["status"][0] == 1
    r = oracle.render(s)
    assert r["stats"]["visible"] == 1
    assert r["count"].max() == 1
