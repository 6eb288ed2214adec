"""Hand-built test scenes (no rasterisation arithmetic here: geometry and colours only)."""
from __future__ import annotations

import numpy as np

import scenegen
from scenegen import COLOR_FLAT, COLOR_VERTEX, Scene


def rects_scene(rects, width=16, height=16, colors=None, depths=None, reverse=False,
                rotate=0):
    """Axis-aligned screen rectangles under the pixel pinhole camera.

    rects: list of (x0, y0, x1, y1) in screen pixels; depths: view depth z per rect
    (world coordinates are scaled by z so the screen footprint is unchanged).
    reverse flips the winding; rotate cycles the starting vertex (changes the diagonal).
    """
    m, n, f = scenegen.pixel_pinhole(width, height)
    pos = []
    for i, (x0, y0, x1, y1) in enumerate(rects):
        z = 1.0 if depths is None else depths[i]
        corners = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
        if reverse:
            corners = corners[::-1]
        corners = corners[rotate:] + corners[:rotate]
        pos.extend([(x * z, y * z, z) for x, y in corners])
    pos = np.array(pos, np.float32).reshape(-1, 3)
    q = len(rects)
    if colors is None:
        colors = np.tile(np.array([[0.2, 0.4, 0.6, 0.5]], np.float32), (q, 1))
    return Scene(pos, None, np.asarray(colors, np.float32), COLOR_FLAT, m, float(n), float(f),
                 width, height, name="rects")


def screen_quads_scene(quads_xy, width, height, colors, depth=1.0, indices=None,
                       color_mode=COLOR_FLAT):
    """Arbitrary screen-space quads (or a shared vertex array with indices) at one depth."""
    m, n, f = scenegen.pixel_pinhole(width, height)
    xy = np.asarray(quads_xy, np.float64).reshape(-1, 2)
    pos = np.concatenate([xy * depth, np.full((xy.shape[0], 1), depth)], axis=1).astype(np.float32)
    idx = None if indices is None else np.asarray(indices, np.uint32)
    return Scene(pos, idx, np.asarray(colors, np.float32), color_mode, m, float(n), float(f),
                 width, height, name="screen")


def shared_grid(nx, ny, x0, y0, x1, y1, jitter=0.0, seed=0, exact_centres=False):
    """An nx x ny grid of quads over [x0,x1]x[y0,y1] sharing vertices (screen units).

    jitter moves interior vertices by up to jitter * cell size; exact_centres snaps every
    vertex to a pixel centre (k + 0.5) so edges run through sample points.
    Returns (vertex_xy [V][2], indices [Q][4]).
    """
    rng = np.random.default_rng(seed)
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    gx, gy = np.meshgrid(xs, ys)
    if jitter:
        cw, ch = (x1 - x0) / nx, (y1 - y0) / ny
        jx = rng.uniform(-jitter, jitter, gx.shape) * cw
        jy = rng.uniform(-jitter, jitter, gy.shape) * ch
        jx[0, :] = jx[-1, :] = 0
        jx[:, 0] = jx[:, -1] = 0
        jy[0, :] = jy[-1, :] = 0
        jy[:, 0] = jy[:, -1] = 0
        gx = gx + jx
        gy = gy + jy
    if exact_centres:
        gx = np.floor(gx) + 0.5
        gy = np.floor(gy) + 0.5
    vxy = np.stack([gx, gy], axis=-1).reshape(-1, 2)
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    base = (iy * (nx + 1) + ix).reshape(-1)
    idx = np.stack([base, base + 1, base + nx + 2, base + nx + 1], axis=1)
    return vxy, idx


def permute_scene(scene: Scene, perm):
    """Reorder the quads of a scene: new quad i is old quad perm[i]."""
    perm = np.asarray(perm)
    if scene.indices is not None:
        idx = scene.indices[perm]
        pos = scene.positions
    else:
        pos = scene.positions.reshape(-1, 4, 3)[perm].reshape(-1, 3)
        idx = None
    col = scene.colors[perm] if scene.color_mode == COLOR_FLAT else scene.colors
    return Scene(np.ascontiguousarray(pos), None if idx is None else np.ascontiguousarray(idx),
                 np.ascontiguousarray(col), scene.color_mode, scene.view_proj, scene.near,
                 scene.far, scene.width, scene.height, name=scene.name + "-perm")


def tilted_plane_quad(width, height, depth, slope_x, slope_y, half, color_mode=COLOR_FLAT,
                      vertex_colors=None, flat_color=(0.3, 0.6, 0.9, 0.5), center=(0.0, 0.0)):
    """One planar quad in the plane z = -(depth + slope_x * x + slope_y * y), perspective camera."""
    m, n, f = scenegen.perspective(width, height)
    cx, cy = center
    pts = []
    for sx, sy in ((-1, -1), (1, -1), (1, 1), (-1, 1)):
        x, y = cx + sx * half, cy + sy * half
        pts.append((x, y, -(depth + slope_x * x + slope_y * y)))
    pos = np.array(pts, np.float32)
    if color_mode == COLOR_FLAT:
        col = np.array([flat_color], np.float32)
    else:
        col = np.asarray(vertex_colors, np.float32)
    return Scene(pos, None, col, color_mode, m, float(n), float(f), width, height, name="tilted")


def concat_scenes(a: Scene, b: Scene) -> Scene:
    """Concatenate two non-indexed flat scenes that share a camera."""
    assert a.indices is None and b.indices is None
    assert a.color_mode == b.color_mode == COLOR_FLAT
    return Scene(np.concatenate([a.positions, b.positions]), None,
                 np.concatenate([a.colors, b.colors]), COLOR_FLAT, a.view_proj, a.near, a.far,
                 a.width, a.height, name=a.name + "+" + b.name)
