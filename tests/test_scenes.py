"""The seeded generators produce the workload shapes the benchmarks and parity tests use."""
import numpy as np

import scenegen


def test_small_frustum_shape():
    s = scenegen.config_small_frustum()
    assert s.num_quads == 2000 and s.indices is None and s.positions.shape == (8000, 3)
    assert s.colors.shape == (2000, 4) and s.color_mode == scenegen.COLOR_FLAT
    a = s.colors[:, 3]
    assert a.min() >= 0.2 and a.max() <= 0.8
    # deterministic
    np.testing.assert_array_equal(s.positions, scenegen.config_small_frustum().positions)


def test_layers_shape():
    s = scenegen.wavy_layers(1920, 1080, 32, 256, 128)
    assert s.num_quads == 1_048_576 and s.num_vertices == 32 * 257 * 129
    assert s.indices.max() < s.num_vertices
    assert s.colors.shape == (s.num_vertices, 4)
    assert s.colors[:, 3].min() >= 0.1 and s.colors[:, 3].max() <= 0.5


def test_particles_shape():
    s = scenegen.gaussian_particles(10_000, 1920, 1080, seed=3)
    assert s.num_quads == 10_000 and s.positions.shape == (40_000, 3)
    q = s.positions.reshape(-1, 4, 3)
    # camera-facing: the four corners share one depth
    assert np.all(q[:, :, 2] == q[:, :1, 2])


def test_request_trace():
    tr = scenegen.request_trace(256, 200.0, seed=0)
    assert len(tr) == 256
    t = np.array([r["arrival"] for r in tr])
    assert np.all(np.diff(t) >= 0) and t[0] == 0.0
    assert 0.8 < 255 / t[-1] / 200.0 < 1.25
    assert {(r["width"], r["height"]) for r in tr} <= set(scenegen.RESOLUTIONS)
    assert all(10_000 <= r["quads"] <= 2_000_000 for r in tr)


def test_lit_layers_normals_are_the_surface_normals():
    # same geometry and RGBA as the per-vertex scene; the normals are unit length and
    # perpendicular to the displaced surface (checked against central differences of the
    # generated vertex grid)
    nx, ny = 640, 320      # fine enough that central differences are within 1e-3 of the slope
    lit = scenegen.wavy_layers(320, 160, layers=3, nx=nx, ny=ny, seed=4, color_mode=scenegen.COLOR_LIT)
    vtx = scenegen.wavy_layers(320, 160, layers=3, nx=nx, ny=ny, seed=4)
    np.testing.assert_array_equal(lit.positions, vtx.positions)
    np.testing.assert_array_equal(lit.colors[:, :4], vtx.colors)
    assert lit.colors.shape == (lit.num_vertices, 8) and lit.light is not None
    n = lit.colors[:, 4:7].astype(np.float64)
    assert np.abs(np.linalg.norm(n, axis=1) - 1).max() < 1e-6
    p = lit.positions.astype(np.float64).reshape(3, ny + 1, nx + 1, 3)
    nl = n.reshape(3, ny + 1, nx + 1, 3)
    tx = p[:, 1:-1, 2:, :] - p[:, 1:-1, :-2, :]      # along the grid's x
    ty = p[:, 2:, 1:-1, :] - p[:, :-2, 1:-1, :]      # along the grid's y
    ni = nl[:, 1:-1, 1:-1, :]
    for t in (tx, ty):
        cos = np.abs(np.sum(t * ni, axis=-1)) / np.linalg.norm(t, axis=-1)
        assert cos.max() < 2e-3                    # (second order: 0.19 at 40 cells, 0.011 at 160)
    assert np.all(ni[..., 2] > 0)                    # facing the camera side (+z)
