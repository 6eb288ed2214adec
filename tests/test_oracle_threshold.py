"""Pins of the oracle's opt-in alpha-threshold composite (Sec. 2, "Sample blending": with
the 'alpha_threshold' flag, shading and blending stop once the accumulated alpha reaches
1 - 1/128; Sec. 3, "Alpha threshold"). The mode is lossy by design; these checks pin the
stop rule with closed forms, its limit t_min = 0, its error bound against the exact
composite, and its independence of submission order."""
import numpy as np
import pytest

import oracle
import scenegen
from scenegen import COLOR_FLAT
from tests.scene_helpers import permute_scene, rects_scene

T_MIN = 1.0 / 128.0


def _stack(alpha, layers=10):
    rng = np.random.default_rng(3)
    cols = np.concatenate([rng.random((layers, 3)), np.full((layers, 1), alpha)], 1).astype(np.float32)
    depths = [1.0 + 0.25 * k for k in range(layers)]          # layer 0 is the nearest
    s = rects_scene([(2, 2, 10, 10)] * layers, depths=depths, colors=cols)
    return s, cols


@pytest.mark.parametrize("alpha,blended", [(0.5, 7), (0.75, 4)])
def test_stack_closed_form(alpha, blended):
    # T before the k-th nearest layer is (1 - a)^k, a power of two here, so every stop
    # test is exact: with a = 1/2 the 8th layer meets T = 1/128 and is the first dropped;
    # with a = 3/4 the 5th meets T = 1/256
    s, cols = _stack(alpha)
    r = oracle.render_threshold(s, T_MIN)
    assert np.all(r["nblend"][2:10, 2:10] == blended)
    assert np.all(r["count"][2:10, 2:10] == 10)
    want = np.zeros(3)
    for k in range(blended):
        want += (1 - alpha) ** k * alpha * cols[k, :3].astype(np.float64)
    got = r["rgba"][5, 5].astype(np.float64)
    assert np.abs(got[:3] - want).max() < 1e-7
    assert got[3] == 1.0 - (1 - alpha) ** blended
    # outside the stack nothing is drawn
    assert np.all(r["rgba"][0, 0] == 0) and r["nblend"][0, 0] == 0


def test_stop_test_is_inclusive():
    # T = 1/128 exactly stops (accumulated alpha "at least" 1 - 1/128); a threshold just
    # below lets the 8th layer through
    s, _ = _stack(0.5)
    assert oracle.render_threshold(s, T_MIN)["nblend"][5, 5] == 7
    assert oracle.render_threshold(s, np.nextafter(np.float32(T_MIN), np.float32(0)))["nblend"][5, 5] == 8


def _dense_scenes():
    return [scenegen.wavy_layers(96, 64, layers=32, nx=12, ny=8, seed=1),
            scenegen.wavy_layers(64, 48, layers=32, nx=10, ny=8, seed=4, color_mode=COLOR_FLAT),
            scenegen.gaussian_particles(6000, 96, 64, seed=2)]


@pytest.mark.parametrize("k", range(3))
def test_zero_threshold_is_the_exact_composite(k):
    s = _dense_scenes()[k]
    exact = oracle.render(s)
    r = oracle.render_threshold(s, 0.0)
    np.testing.assert_array_equal(r["nblend"], exact["count"])
    assert np.abs(r["rgba"].astype(np.float64) - exact["rgba"]).max() < 2e-6


@pytest.mark.parametrize("k", range(3))
def test_error_bound_against_exact(k):
    # the dropped fragments sit behind a transmittance T <= t_min and their composite is
    # at most 1 per channel, so the image moves by at most t_min
    s = _dense_scenes()[k]
    exact = oracle.render(s)
    r = oracle.render_threshold(s, T_MIN)
    err = np.abs(r["rgba"].astype(np.float64) - exact["rgba"].astype(np.float64))
    assert err.max() <= T_MIN + 2e-6
    nb, cnt = r["nblend"], exact["count"]
    assert np.all(nb <= cnt)
    cut = nb < cnt
    assert cut.sum() > 0.05 * cnt.size          # the scenes are deep enough to saturate
    # stopped pixels reached the threshold; complete pixels match the exact composite
    assert np.all(1.0 - r["rgba"][..., 3][cut] <= T_MIN * (1 + 1e-6))
    assert err[~cut].max() < 2e-6


def test_stop_index_from_the_pixel_fragment_lists():
    # the sorted fragment list of a pixel (an enumeration separate from the image pass)
    # walked front to back with fp32 transmittance gives the same number blended
    s = _dense_scenes()[0]
    r = oracle.render_threshold(s, T_MIN)
    rng = np.random.default_rng(5)
    for _ in range(40):
        px, py = int(rng.integers(0, s.width)), int(rng.integers(0, s.height))
        fr = oracle.pixel_fragments(s, px, py)
        T = np.float32(1.0)
        n = 0
        for a in fr["rgba"][::-1, 3]:
            if not T > np.float32(T_MIN):
                break
            T = np.float32(T * np.float32(np.float32(1.0) - a))
            n += 1
        assert n == r["nblend"][py, px], (px, py)


def test_threshold_image_independent_of_submission_order():
    s = _dense_scenes()[1]
    r0 = oracle.render_threshold(s, T_MIN)
    perm = np.random.default_rng(11).permutation(s.num_quads)
    r1 = oracle.render_threshold(permute_scene(s, perm), T_MIN)
    np.testing.assert_array_equal(r0["rgba"], r1["rgba"])
    np.testing.assert_array_equal(r0["nblend"], r1["nblend"])
