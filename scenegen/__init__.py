"""Seeded synthetic scene generators shared by the CUDA path's tests/bench and the oracle.

This module holds no rasterisation arithmetic: it only draws random quads, colours and
cameras with ``numpy.random.default_rng`` (PCG64) and returns plain numpy arrays.
Both sides are fed the same arrays, so neither re-implements the random stream.

The paper's 12 test scenes (Sec. 3, "Test scenes") are not available; the generators
below stand in for them with the shapes, sizes and depth structure of the workloads
the pipeline is measured on (a frustum of random parallelograms, stacked wavy
transparent layers with perspective-correct vertex colours, and a dense particle cloud).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

COLOR_FLAT = 0
COLOR_VERTEX = 1
COLOR_LIT = 2       # per-vertex [V][8]: straight RGBA, unit normal xyz, unused

# Half-height (world units) of a layer of the stacked-layer generator, calibrated so
# that 32 layers at view depths 2.0, 2.5, ..., 17.5 give a mean depth complexity of
# about 24 (analytic footprint sum, checked against measured fragment counts).
LAYER_HALF_H_WIDE = 5.09    # 16:9 screen, layer half-width = 2 x half-height
LAYER_HALF_H_SQUARE = 5.38  # 1:1 screen, layer half-width = half-height


@dataclasses.dataclass
class Scene:
    """A quad scene plus camera, all host numpy arrays.

    positions  f32[V][3]  world-space vertex positions
    indices    u32[Q][4] or None (None: quad q uses vertices 4q..4q+3)
    colors     f32[Q][4] (flat, straight RGBA) or f32[V][4] (per-vertex)
    color_mode COLOR_FLAT | COLOR_VERTEX
    view_proj  f32[4][4]  row-major; clip = view_proj @ (x, y, z, 1); clip.w = view depth
    near, far  clip.w range a quad's vertices must lie in
    width, height  target resolution in pixels
    """

    positions: np.ndarray
    indices: np.ndarray | None
    colors: np.ndarray
    color_mode: int
    view_proj: np.ndarray
    near: float
    far: float
    width: int
    height: int
    name: str = ""
    light: tuple | None = None   # lit colours: (x, y, z) toward the light (world), ambient

    @property
    def num_quads(self) -> int:
        if self.indices is not None:
            return int(self.indices.shape[0])
        return int(self.positions.shape[0] // 4)

    @property
    def num_vertices(self) -> int:
        return int(self.positions.shape[0])

    def with_colors(self, colors: np.ndarray) -> "Scene":
        return dataclasses.replace(self, colors=np.ascontiguousarray(colors, np.float32))


def perspective(width: int, height: int, fovy_deg: float = 60.0,
                near: float = 0.1, far: float = 100.0):
    """Row-major view-projection of a camera at the origin looking down -z.

    Row 3 is (0, 0, -1, 0) so clip.w = -z = view depth. Row 2 is the usual OpenGL
    depth row; the rasteriser does not read it.
    """
    aspect = width / height
    f = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    m = np.zeros((4, 4), np.float64)
    m[0, 0] = f / aspect
    m[1, 1] = f
    m[2, 2] = -(far + near) / (far - near)
    m[2, 3] = -2.0 * far * near / (far - near)
    m[3, 2] = -1.0
    return m.astype(np.float32), np.float32(near), np.float32(far)


def pixel_pinhole(width: int, height: int, near: float = 0.5, far: float = 4.0):
    """A pinhole camera that maps world (x, y, z), z > 0, to screen pixel (x/z, y/z).

    Rows: (2/W, 0, -1, 0), (0, -2/H, 1, 0), unused, (0, 0, 1, 0), so clip.w = z and
    the screen position (row 0 at the top) is exactly (x/z, y/z) whenever the fp32
    arithmetic is exact, e.g. for power-of-two W, H, z in {1, 2} and short binary
    fractions. Used by the closed-form tests.
    """
    m = np.zeros((4, 4), np.float32)
    m[0, 0] = 2.0 / width
    m[0, 2] = -1.0
    m[1, 1] = -2.0 / height
    m[1, 2] = 1.0
    m[3, 2] = 1.0
    return m, np.float32(near), np.float32(far)


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def frustum_parallelograms(num_quads: int = 2000, width: int = 256, height: int = 256,
                           seed: int = 0, fovy_deg: float = 60.0, near: float = 0.1,
                           far: float = 100.0, edge_range=(0.05, 1.5),
                           alpha_range=(0.2, 0.8)) -> Scene:
    """Planar parallelograms with centres uniform in the view frustum's volume.

    Depth d has density proportional to d^2 on [near, far] (inverse CDF
    d = (n^3 + u (f^3 - n^3))^(1/3)); the centre is then uniform over the frustum's
    cross-section at d. Two edge vectors of length U[edge_range] with independent
    uniform-sphere directions span the quad; vertices c -/+ e1/2 -/+ e2/2.
    Flat RGBA: RGB U[0,1], A U[alpha_range]. Non-indexed.
    """
    rng = np.random.default_rng(seed)
    m, n, f = perspective(width, height, fovy_deg, near, far)
    t = math.tan(math.radians(fovy_deg) / 2.0)
    aspect = width / height
    u = rng.random(num_quads)
    d = np.cbrt(near ** 3 + u * (far ** 3 - near ** 3))
    cx = (rng.random(num_quads) * 2 - 1) * d * t * aspect
    cy = (rng.random(num_quads) * 2 - 1) * d * t
    c = np.stack([cx, cy, -d], axis=1)
    l1 = rng.uniform(edge_range[0], edge_range[1], num_quads)[:, None]
    l2 = rng.uniform(edge_range[0], edge_range[1], num_quads)[:, None]
    e1 = _unit_vectors(rng, num_quads) * l1
    e2 = _unit_vectors(rng, num_quads) * l2
    v = np.stack([c - e1 / 2 - e2 / 2, c + e1 / 2 - e2 / 2,
                  c + e1 / 2 + e2 / 2, c - e1 / 2 + e2 / 2], axis=1)
    pos = v.reshape(-1, 3).astype(np.float32)
    col = np.empty((num_quads, 4), np.float32)
    col[:, :3] = rng.random((num_quads, 3))
    col[:, 3] = rng.uniform(alpha_range[0], alpha_range[1], num_quads)
    return Scene(pos, None, col, COLOR_FLAT, m, float(n), float(f), width, height,
                 name=f"frustum{num_quads}")


def wavy_layers(width: int = 1920, height: int = 1080, layers: int = 32, nx: int = 256,
                ny: int = 128, seed: int = 0, color_mode: int = COLOR_VERTEX,
                half_h: float | None = None, d0: float = 2.0, dz: float = 0.5,
                amplitude: float = 0.3, alpha_range=(0.1, 0.5)) -> Scene:
    """Stacked transparent layers, each an nx x ny grid of quads displaced by 4 sines.

    Layer k lies at view depth d0 + dz*k; a vertex (x, y) of layer k is moved along
    view z by sum_m amplitude * sin(k_m . (x, y) + phi_m), m = 1..4, with |k_m| U[0.5, 3]
    rad/unit, a uniform direction and phi_m U[0, 2pi), drawn from default_rng(k).
    Each term has amplitude 0.3, so neighbouring layers can interpenetrate.
    Vertices are shared (indexed quads); colours are per-vertex (perspective-correct)
    or flat per quad, RGB U[0,1], A U[alpha_range], drawn from default_rng(seed).
    """
    m, n, f = perspective(width, height)
    aspect = width / height
    if half_h is None:
        half_h = LAYER_HALF_H_WIDE if aspect > 1.2 else LAYER_HALF_H_SQUARE
    half_w = half_h * nx / ny
    xs = np.linspace(-half_w, half_w, nx + 1)
    ys = np.linspace(-half_h, half_h, ny + 1)
    gx, gy = np.meshgrid(xs, ys)  # [ny+1][nx+1]
    verts = []
    normals = []
    for k in range(layers):
        lr = np.random.default_rng(k)
        kmag = lr.uniform(0.5, 3.0, 4)
        ang = lr.uniform(0.0, 2 * np.pi, 4)
        phi = lr.uniform(0.0, 2 * np.pi, 4)
        disp = np.zeros_like(gx)
        for i in range(4):
            disp += amplitude * np.sin(kmag[i] * (np.cos(ang[i]) * gx + np.sin(ang[i]) * gy) + phi[i])
        z = -(d0 + dz * k) + disp
        verts.append(np.stack([gx, gy, z], axis=-1).reshape(-1, 3))
        if color_mode == COLOR_LIT:
            # the displaced surface's unit normal (-dz/dx, -dz/dy, 1) / norm
            dzx = np.zeros_like(gx)
            dzy = np.zeros_like(gx)
            for i in range(4):
                c = amplitude * kmag[i] * np.cos(kmag[i] * (np.cos(ang[i]) * gx + np.sin(ang[i]) * gy) + phi[i])
                dzx += c * np.cos(ang[i])
                dzy += c * np.sin(ang[i])
            nrm = np.stack([-dzx, -dzy, np.ones_like(gx)], axis=-1).reshape(-1, 3)
            normals.append(nrm / np.linalg.norm(nrm, axis=1, keepdims=True))
    pos = np.concatenate(verts).astype(np.float32)
    nvl = (nx + 1) * (ny + 1)
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    base = (iy * (nx + 1) + ix).reshape(-1)
    quad = np.stack([base, base + 1, base + nx + 2, base + nx + 1], axis=1)
    idx = np.concatenate([quad + k * nvl for k in range(layers)]).astype(np.uint32)
    rng = np.random.default_rng(seed)
    count = pos.shape[0] if color_mode in (COLOR_VERTEX, COLOR_LIT) else idx.shape[0]
    col = np.empty((count, 4), np.float32)
    col[:, :3] = rng.random((count, 3))
    col[:, 3] = rng.uniform(alpha_range[0], alpha_range[1], count)
    light = None
    if color_mode == COLOR_LIT:
        lit = np.zeros((count, 8), np.float32)
        lit[:, :4] = col
        lit[:, 4:7] = np.concatenate(normals)
        col = lit
        light = (0.4, 0.6, 1.0, 0.25)
    return Scene(pos, idx, col, color_mode, m, float(n), float(f), width, height,
                 name=f"layers{layers}x{nx}x{ny}", light=light)


def gaussian_particles(num_quads: int = 2_000_000, width: int = 1920, height: int = 1080,
                       seed: int = 0, center_depth: float = 10.0, sigma: float = 2.0,
                       size_px=(2.0, 16.0), alpha_range=(0.02, 0.3)) -> Scene:
    """Camera-facing squares, 2-16 px on screen, centres ~ N((0,0,-10), sigma^2 I).

    Side s_px ~ U[size_px] is converted to world units at the centre's depth d:
    s = s_px * 2 d tan(30 deg) / height, so every quad lies in a plane of constant depth.
    Flat RGBA: RGB U[0,1], A U[alpha_range]. Non-indexed.
    """
    rng = np.random.default_rng(seed)
    m, n, f = perspective(width, height)
    c = rng.standard_normal((num_quads, 3)) * sigma
    c[:, 2] -= center_depth
    d = -c[:, 2]
    s_px = rng.uniform(size_px[0], size_px[1], num_quads)
    s = s_px * 2.0 * d * math.tan(math.radians(30.0)) / height
    h = (s / 2.0)[:, None]
    ex = np.array([1.0, 0.0, 0.0])[None, :]
    ey = np.array([0.0, 1.0, 0.0])[None, :]
    v = np.stack([c - h * ex - h * ey, c + h * ex - h * ey,
                  c + h * ex + h * ey, c - h * ex + h * ey], axis=1)
    pos = v.reshape(-1, 3).astype(np.float32)
    col = np.empty((num_quads, 4), np.float32)
    col[:, :3] = rng.random((num_quads, 3))
    col[:, 3] = rng.uniform(alpha_range[0], alpha_range[1], num_quads)
    return Scene(pos, None, col, COLOR_FLAT, m, float(n), float(f), width, height,
                 name=f"particles{num_quads}")


def perturbed_target_colors(colors: np.ndarray, seed: int = 1, sigma: float = 0.05):
    """Per-quad RGBA + N(0, sigma), clamped to [0, 1] (the differentiable-compositing target)."""
    rng = np.random.default_rng(seed)
    return np.clip(colors + rng.normal(0.0, sigma, colors.shape), 0.0, 1.0).astype(np.float32)


# ---- the named workloads -------------------------------------------------------------

def config_small_frustum(seed: int = 0) -> Scene:
    """256x256, 2,000 random parallelograms, flat RGBA (the oracle-parity case)."""
    return frustum_parallelograms(2000, 256, 256, seed=seed)


def config_layers_1080p(seed: int = 0) -> Scene:
    """1920x1080, 32 layers x 256x128 quads = 1,048,576 quads, per-vertex RGBA."""
    return wavy_layers(1920, 1080, 32, 256, 128, seed=seed, color_mode=COLOR_VERTEX)


def config_particles_1080p(seed: int = 0) -> Scene:
    """1920x1080, 2,000,000 camera-facing particles, flat RGBA, centre depth > 500."""
    return gaussian_particles(2_000_000, 1920, 1080, seed=seed)


def config_diff_1024(seed: int = 0) -> Scene:
    """1024x1024, 32 layers x 128x128 = 524,288 quads, flat per-quad RGBA."""
    return wavy_layers(1024, 1024, 32, 128, 128, seed=seed, color_mode=COLOR_FLAT)


RESOLUTIONS = [(256, 256), (1024, 768), (1920, 1080), (2560, 1440)]


def request_trace(num_requests: int = 256, rate_hz: float = 200.0, seed: int = 0,
                  min_quads: int = 10_000, max_quads: int = 2_000_000):
    """Poisson arrivals (exponential gaps) of render requests of mixed size.

    Each request: arrival time (s), resolution from RESOLUTIONS, generator kind
    ('frustum' | 'layers' | 'particles') and a quad count log-uniform in
    [min_quads, max_quads]. Scenes are built later with ``scene_for_request``.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, num_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(num_requests):
        w, h = RESOLUTIONS[int(rng.integers(len(RESOLUTIONS)))]
        kind = ("frustum", "layers", "particles")[int(rng.integers(3))]
        q = int(round(math.exp(rng.uniform(math.log(min_quads), math.log(max_quads)))))
        out.append(dict(id=i, arrival=float(t[i]), width=w, height=h, kind=kind,
                        quads=q, seed=1000 + i))
    return out


def scene_for_request(req) -> Scene:
    """Build the scene a trace entry describes (layers: grid scaled to the quad count)."""
    kind, q, w, h, seed = req["kind"], req["quads"], req["width"], req["height"], req["seed"]
    if kind == "frustum":
        return frustum_parallelograms(q, w, h, seed=seed)
    if kind == "particles":
        return gaussian_particles(q, w, h, seed=seed)
    per_layer = max(1, q // 32)
    ny = max(1, int(round(math.sqrt(per_layer / 2.0))))
    nx = max(1, per_layer // ny)
    return wavy_layers(w, h, 32, nx, ny, seed=seed, color_mode=COLOR_VERTEX)
