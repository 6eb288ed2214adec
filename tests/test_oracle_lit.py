"""Pins of the oracle's lit colour mode: per-vertex normals and one directional light
(the paper shades its samples with a simple material, Sec. 2 "Stage 3" and Sec. 4; its
shaders and textures are not available, so this is the plainest shading with normals:
two-sided Lambert plus ambient on the perspective-correct base colour)."""
import dataclasses

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import COLOR_LIT, COLOR_VERTEX
from tests.scene_helpers import rects_scene, tilted_plane_quad

LIGHT = (0.4, 0.6, 1.0, 0.25)


def _lit_layers(**kw):
    return scenegen.wavy_layers(96, 64, layers=8, nx=12, ny=8, seed=1, color_mode=COLOR_LIT, **kw)


def _with(scene, colors=None, light=None):
    return dataclasses.replace(scene, colors=scene.colors if colors is None else
                               np.ascontiguousarray(colors, np.float32),
                               light=scene.light if light is None else light)


def test_full_ambient_is_the_vertex_colour_image():
    s = _lit_layers()
    lit = oracle.render(_with(s, light=(0.4, 0.6, 1.0, 1.0)))["rgba"]
    v = dataclasses.replace(s, colors=np.ascontiguousarray(s.colors[:, :4]), color_mode=COLOR_VERTEX, light=None)
    np.testing.assert_array_equal(lit, oracle.render(v)["rgba"])


def _one_rect_lit(normals, base=(0.8, 0.6, 0.4, 0.5), light=LIGHT):
    s = rects_scene([(2, 2, 12, 10)], width=16, height=12)
    col = np.zeros((4, 8), np.float32)
    col[:, :4] = base
    col[:, 4:7] = normals
    return dataclasses.replace(s, colors=col, color_mode=COLOR_LIT, light=light)


def test_constant_normal_closed_form():
    n = np.array([0.3, -0.5, 0.8])
    s = _one_rect_lit(np.tile(n, (4, 1)))
    r = oracle.render(s)["rgba"]
    L = np.array(LIGHT[:3])
    f = LIGHT[3] + (1 - LIGHT[3]) * abs(n @ L) / (np.linalg.norm(n) * np.linalg.norm(L))
    base = np.array([0.8, 0.6, 0.4])
    want = 0.5 * base * f
    assert np.abs(r[5, 5, :3] - want).max() < 1e-6
    assert abs(r[5, 5, 3] - 0.5) < 1e-7
    assert np.all(r[0, 0] == 0)


def test_normal_interpolation_on_a_tilted_quad():
    # the perspective-correct normal is the screen-space rational fit (sum q n) / (sum q)
    # through the snapped vertices; its direction sets the Lambert term
    nv = np.array([[1.0, 0.0, 0.2], [0.0, 1.0, 0.3], [-0.6, 0.2, 1.0], [0.3, -0.8, 0.5]])
    col = np.zeros((4, 8), np.float32)
    col[:, :4] = (0.9, 0.7, 0.5, 0.6)
    col[:, 4:7] = nv
    s = tilted_plane_quad(64, 64, depth=2.0, slope_x=1.5, slope_y=0.3, half=1.0, color_mode=COLOR_LIT,
                          vertex_colors=col)
    s = dataclasses.replace(s, light=LIGHT)
    st = oracle.setup(s)
    X = st["X"][0].astype(np.float64) / 256.0
    Y = st["Y"][0].astype(np.float64) / 256.0
    q = st["q"][0].astype(np.float64)
    L = np.array(LIGHT[:3]) / np.linalg.norm(LIGHT[:3])
    checked = 0
    for t, (a, b, c) in enumerate(((0, 1, 2), (0, 2, 3))):
        A = np.array([[X[a], Y[a], 1.0], [X[b], Y[b], 1.0], [X[c], Y[c], 1.0]])
        num = np.linalg.solve(A, q[[a, b, c], None] * nv[[a, b, c]])
        for py in range(0, 64, 4):
            for px in range(0, 64, 4):
                fr = oracle.pixel_fragments(s, px, py)
                for rgba, tri in zip(fr["rgba"], fr["tri"]):
                    if tri != t:
                        continue
                    n = np.array([px + 0.5, py + 0.5, 1.0]) @ num
                    f = LIGHT[3] + (1 - LIGHT[3]) * abs(n @ L) / np.linalg.norm(n)
                    want = np.array([0.9, 0.7, 0.5]) * f
                    assert np.abs(rgba[:3] - want).max() < 2e-6
                    checked += 1
    assert checked > 20


@pytest.mark.parametrize("change", ["scale_normals", "negate_normals", "scale_light", "rotate_both"])
def test_lighting_invariances(change):
    s = _lit_layers()
    base = oracle.render(s)["rgba"]
    col = s.colors.copy()
    light = s.light
    if change == "scale_normals":
        col[:, 4:7] *= 3.5
    elif change == "negate_normals":       # two-sided: the back face is lit the same
        col[:, 4:7] *= -1.0
    elif change == "scale_light":
        light = tuple(2.5 * v for v in light[:3]) + (light[3],)
    else:                                   # the same rotation of normals and light
        th = 0.7
        R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
        col[:, 4:7] = (col[:, 4:7].astype(np.float64) @ R.T).astype(np.float32)
        light = tuple(float(v) for v in (R @ np.array(light[:3]))) + (light[3],)
    got = oracle.render(_with(s, colors=col, light=light))["rgba"]
    assert np.abs(got - base).max() < 2e-6


def test_lit_is_never_brighter_than_unlit():
    s = _lit_layers()
    lit = oracle.render(s)["rgba"]
    v = dataclasses.replace(s, colors=np.ascontiguousarray(s.colors[:, :4]), color_mode=COLOR_VERTEX, light=None)
    un = oracle.render(v)["rgba"]
    assert np.all(lit[..., :3] <= un[..., :3] + 1e-7)
    np.testing.assert_array_equal(lit[..., 3], un[..., 3])
    assert lit[..., :3].mean() < 0.95 * un[..., :3].mean()
