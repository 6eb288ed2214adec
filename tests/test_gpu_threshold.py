"""GPU parity of the opt-in alpha-threshold composite (LR_FLAG_ALPHA_THRESHOLD; Sec. 2,
"Sample blending": blending stops once a pixel's accumulated alpha reaches 1 - 1/128;
Sec. 3, "Alpha threshold") with the oracle's threshold composite. Every call goes
through the C ABI via the ctypes binding.

Bar. With flat per-quad alpha the stop decision is fixed by exact inputs: both sides form
the same fp32 running product of (1 - a) in the same exact depth order, so every pixel
must be within 1e-5 of the oracle's threshold composite. With per-vertex colours the
interpolated alpha is rounded differently on the two sides, so a pixel whose
transmittance passes within 1e-3 (relative) of 1/128 at a stop test may stop one
fragment earlier or later there: such pixels (a few percent at most) must instead meet
the bound both stops satisfy, the exact composite within 1/128 (plus rounding); all
other pixels within 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from scenegen import COLOR_FLAT
from tests.scene_helpers import rects_scene

pytestmark = pytest.mark.gpu

T_MIN = 1.0 / 128.0
COLOR_TOL = 1e-5
AMBIGUOUS = 1e-3


@pytest.fixture(scope="module")
def lr():
    import paper_2405_13364_gb300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    P.load_library()
    return P


_renderers = {}


def renderer(lr, k):
    if k not in _renderers:
        _renderers[k] = lr.Renderer(sorter_k=k, alpha_threshold=True)
    return _renderers[k]


def render_threshold(lr, scene, k):
    r = renderer(lr, k)
    out = r.render(lr.DeviceScene.from_scene(scene), scene.width, scene.height)
    torch.cuda.synchronize()
    return out["rgba"].cpu().numpy(), r.stats()


def stack_scene():
    rng = np.random.default_rng(3)
    cols = np.concatenate([rng.random((10, 3)), np.full((10, 1), 0.5)], 1).astype(np.float32)
    return rects_scene([(2, 2, 30, 20)] * 10, width=40, height=24,
                       depths=[1.0 + 0.25 * k for k in range(10)], colors=cols)


def scenes():
    return {
        "stack": stack_scene(),
        "layers_flat": scenegen.wavy_layers(256, 256, layers=24, nx=32, ny=32, seed=2,
                                            color_mode=COLOR_FLAT),
        "layers_vertex": scenegen.wavy_layers(333, 190, layers=32, nx=48, ny=24, seed=1),
        "particles": scenegen.gaussian_particles(60_000, 320, 180, seed=3),
    }


def assert_threshold_parity(g, scene):
    o = oracle.render_threshold(scene, T_MIN)
    if scene.color_mode == COLOR_FLAT:
        amb = np.zeros(o["margin"].shape, bool)
    else:
        amb = o["margin"] < AMBIGUOUS
    d = np.abs(g.astype(np.float64) - o["rgba"].astype(np.float64))
    assert d[~amb].max() <= COLOR_TOL, f"max error {d[~amb].max()}"
    assert amb.mean() < 0.03
    if amb.any():
        exact = oracle.render(scene)["rgba"].astype(np.float64)
        assert np.abs(g[amb].astype(np.float64) - exact[amb]).max() <= T_MIN * (1 + AMBIGUOUS) + COLOR_TOL
    return o


@pytest.mark.parametrize("name", list(scenes()))
@pytest.mark.parametrize("k", [1, 3, 8])
def test_threshold_matches_oracle(lr, name, k):
    scene = scenes()[name]
    g, st = render_threshold(lr, scene, k)
    assert st["status"] == 0
    o = assert_threshold_parity(g, scene)
    if name == "stack":
        assert np.all(o["nblend"][2:20, 2:30] == 7)
    if name == "particles":
        # candidates behind every finished pixel of a half-block were skipped
        assert st["fragments"] < int(o["count"].sum())


def test_threshold_full_size_layers(lr):
    # the 1920x1080 layer frame (1M quads, per-vertex colour) in the bench's configuration
    scene = scenegen.config_layers_1080p()
    g, st = render_threshold(lr, scene, 1)
    assert st["status"] == 0
    assert_threshold_parity(g, scene)


def test_threshold_full_size_particles(lr):
    # the 1920x1080 particle frame (2M quads, flat colour, depth complexity > 500)
    scene = scenegen.config_particles_1080p()
    g, st = render_threshold(lr, scene, 1)
    assert st["status"] == 0
    o = assert_threshold_parity(g, scene)
    assert st["fragments"] < int(o["count"].sum())


def test_threshold_refuses_exact_only_outputs(lr):
    from paper_2405_13364_gb300 import _binding as B
    scene = scenes()["stack"]
    r = renderer(lr, 3)
    ds = lr.DeviceScene.from_scene(scene)
    with pytest.raises(B.LrError) as e:
        r.render(ds, scene.width, scene.height, count=True)
    assert e.value.status == B.LR_ERR_UNSUPPORTED
    fwd = torch.zeros((scene.height, scene.width, 4), dtype=torch.float32, device="cuda")
    grad = torch.zeros_like(fwd)
    gcol = torch.zeros((scene.num_quads, 4), dtype=torch.float32, device="cuda")
    ptr, nbytes = r.workspace(B.lr_workspace_size(r.ctx, ds.num_quads, scene.width, scene.height))
    with pytest.raises(B.LrError) as e:
        B.lr_render_backward(r.ctx, ds.quads_struct(), ds.camera_struct(), scene.width, scene.height,
                             int(fwd.data_ptr()), int(grad.data_ptr()), None, int(gcol.data_ptr()),
                             ptr, nbytes, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == B.LR_ERR_UNSUPPORTED
