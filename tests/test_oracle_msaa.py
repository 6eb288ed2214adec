"""Pins of the oracle's multisampled composite. The paper names 4x and 16x multisample
anti-aliasing as an extension that mainly changes the coverage and blending phases of the
raster stage (Sec. 4, "Future work"). The definition used here: every sample position of
a pixel gets the exact composite of its own covering fragments (coverage, depth key and
colour taken at the sample), and the pixel is the mean of its samples."""
import numpy as np
import pytest

import oracle
from oracle import brute
from tests.scene_helpers import permute_scene, rects_scene
from tests.test_oracle_pins import _tiny_scenes


@pytest.mark.parametrize("n", [4, 16])
def test_patterns_are_n_rooks_inside_the_pixel(n):
    offs = oracle.MSAA_OFFSETS[n]
    assert len(offs) == n and len(set(offs)) == n
    xs = sorted(dx for dx, _ in offs)
    ys = sorted(dy for _, dy in offs)
    # one sample per row and per column of an n x n sub-grid, all strictly inside
    assert len(set(xs)) == n and len(set(ys)) == n
    assert all(-128 < v < 128 for v in xs + ys)
    assert abs(sum(xs)) == 0 and abs(sum(ys)) == 0


@pytest.mark.parametrize("n", [4, 16])
def test_partial_coverage_closed_form(n):
    # a rectangle whose edges cut through pixels: a pixel's value is a c (and a) times the
    # fraction of its samples inside [x0, x1) x [y0, y1) (left and top edges owned)
    x0, y0, x1, y1 = 2 + 77 / 256, 1 + 200 / 256, 9 + 31 / 256, 6 + 128 / 256
    col = np.array([[0.3, 0.7, 0.9, 0.6]], np.float32)
    s = rects_scene([(x0, y0, x1, y1)], width=12, height=9, colors=col)
    got, _ = oracle.render_msaa(s, n)
    offs = oracle.MSAA_OFFSETS[n]
    ac = np.append(col[0, :3] * col[0, 3], col[0, 3]).astype(np.float32)
    seen = set()
    for py in range(s.height):
        for px in range(s.width):
            acc = np.zeros(4, np.float32)
            k = 0
            for dx, dy in offs:
                sx, sy = 256 * px + 128 + dx, 256 * py + 128 + dy
                inside = 256 * x0 <= sx < 256 * x1 and 256 * y0 <= sy < 256 * y1
                k += inside
                acc = (acc + (ac if inside else 0)).astype(np.float32)
            want = acc / np.float32(n)
            assert np.abs(got[py, px] - want).max() <= 1e-7, (px, py)
            seen.add(k)
    assert 0 in seen and n in seen and len(seen) > 2      # partial pixels exist


def test_centre_sample_alone_is_the_plain_image():
    s = _tiny_scenes()[7]
    got, _ = oracle.render_msaa(s, [(0, 0)])
    np.testing.assert_array_equal(got, oracle.render(s)["rgba"])


@pytest.mark.parametrize("k", [0, 3, 6, 7, 8])
def test_brute_force_at_sample_positions(k):
    s = _tiny_scenes()[k]
    for dx, dy in oracle.MSAA_OFFSETS[4][:2] + [(-120, 104)]:
        r = oracle.render(s, sample=(128 + dx, 128 + dy))
        rgba, count, hsh = brute.render(s, sample=(128 + dx, 128 + dy))
        np.testing.assert_array_equal(r["count"], count)
        np.testing.assert_array_equal(r["hash"], hsh)
        np.testing.assert_array_equal(r["rgba"], rgba)


def test_interior_of_parallel_layers_equals_the_plain_image():
    # screen-parallel flat rectangles: every sample of an interior pixel sees the same
    # fragments in the same order, so the mean reproduces the plain pixel
    cols = np.array([[0.9, 0.2, 0.1, 0.5], [0.1, 0.8, 0.3, 0.4], [0.2, 0.3, 0.9, 0.7]], np.float32)
    s = rects_scene([(1, 1, 14, 10), (4, 3, 18, 14), (2, 6, 12, 15)], width=20, height=16,
                    depths=[1.0, 1.5, 2.0], colors=cols)
    got, _ = oracle.render_msaa(s, 16)
    plain = oracle.render(s)["rgba"]
    interior = np.zeros((16, 20), bool)
    interior[2:14, 2:18] = True
    for x0, y0, x1, y1 in [(1, 1, 14, 10), (4, 3, 18, 14), (2, 6, 12, 15)]:
        for e in (x0, x1):
            interior[:, max(e - 1, 0):e + 1] = False
        for e in (y0, y1):
            interior[max(e - 1, 0):e + 1, :] = False
    assert interior.sum() >= 40
    assert np.abs(got[interior] - plain[interior]).max() <= 2e-7


def test_msaa_independent_of_submission_order():
    s = _tiny_scenes()[8]
    a, _ = oracle.render_msaa(s, 4)
    perm = np.random.default_rng(4).permutation(s.num_quads)
    b, _ = oracle.render_msaa(permute_scene(s, perm), 4)
    np.testing.assert_array_equal(a, b)
