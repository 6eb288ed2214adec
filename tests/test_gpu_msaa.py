"""GPU parity of the multisampled render (lr_render_msaa; the paper names 4x and 16x MSAA
as an extension of its raster stage, Sec. 4 "Future work") with the oracle's multisampled
composite: every sample gets the exact composite of the fragments covering it, the pixel
is the mean of its samples. Bar: linear fp32 RGBA within 1e-5 of the oracle per channel.
Every call goes through the C ABI via the ctypes binding."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from scenegen import COLOR_FLAT

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


def scenes():
    return {
        "frustum256": scenegen.config_small_frustum(),
        "frustum_ragged": scenegen.frustum_parallelograms(3000, 200, 141, seed=4),
        "layers_vertex": scenegen.wavy_layers(333, 190, layers=32, nx=48, ny=24, seed=1),
        "layers_flat": scenegen.wavy_layers(160, 120, layers=24, nx=24, ny=16, seed=2, color_mode=COLOR_FLAT),
        "particles": scenegen.gaussian_particles(60_000, 320, 180, seed=3),
    }


def assert_close(g, o, tol=COLOR_TOL):
    d = np.abs(g.astype(np.float64) - o.astype(np.float64))
    assert d.max() <= tol, f"max colour error {d.max()} at {np.unravel_index(d.argmax(), d.shape)}"


@pytest.mark.parametrize("name", list(scenes()))
@pytest.mark.parametrize("n", [4, 16])
def test_msaa_matches_oracle(lr, name, n):
    scene = scenes()[name]
    r = renderer(lr, 1 if n == 16 else 3)
    out = r.render_msaa(lr.DeviceScene.from_scene(scene), scene.width, scene.height, samples=n)
    torch.cuda.synchronize()
    want, _ = oracle.render_msaa(scene, n)
    assert_close(out.cpu().numpy(), want)
    assert r.stats()["n_views"] == n


def test_explicit_patterns(lr):
    scene = scenes()["frustum_ragged"]
    r = renderer(lr)
    ds = lr.DeviceScene.from_scene(scene)
    # extreme offsets (pixel corners) and an odd sample count
    offs = [(-127, 127), (127, -127), (0, -64)]
    out = r.render_msaa(ds, scene.width, scene.height, samples=3, offsets=offs)
    torch.cuda.synchronize()
    want, _ = oracle.render_msaa(scene, offs)
    assert_close(out.cpu().numpy(), want)
    # one sample at the centre is the plain render, bit for bit
    one = r.render_msaa(ds, scene.width, scene.height, samples=1, offsets=[(0, 0)])
    plain = r.render(ds, scene.width, scene.height)["rgba"]
    torch.cuda.synchronize()
    assert torch.equal(one, plain)


def test_msaa_full_size_layers(lr):
    # the 1920x1080 layer frame (1M quads, per-vertex colour) at 4 samples per pixel
    scene = scenegen.config_layers_1080p()
    r = renderer(lr, 1)
    out = r.render_msaa(lr.DeviceScene.from_scene(scene), scene.width, scene.height, samples=4)
    torch.cuda.synchronize()
    want, _ = oracle.render_msaa(scene, 4)
    assert_close(out.cpu().numpy(), want)


def test_msaa_argument_errors(lr):
    from paper_2405_13364_gb300 import _binding as B
    scene = scenes()["frustum256"]
    r = renderer(lr)
    ds = lr.DeviceScene.from_scene(scene)
    W, H = scene.width, scene.height
    out = torch.zeros((H, W, 4), dtype=torch.float32, device="cuda")
    need = B.lr_workspace_size_msaa(r.ctx, ds.num_quads, W, H, 4)
    ptr, nbytes = r.workspace(need)
    st = torch.cuda.current_stream().cuda_stream

    def call(n, offs, nb=nbytes):
        with pytest.raises(B.LrError) as e:
            B.lr_render_msaa(r.ctx, ds.quads_struct(), ds.camera_struct(), W, H, n, offs, int(out.data_ptr()),
                             ptr, nb, st)
        return e.value.status

    assert call(0, None) == B.LR_ERR_INVALID_ARG
    assert call(17, None) == B.LR_ERR_INVALID_ARG
    assert call(3, None) == B.LR_ERR_INVALID_ARG            # no default pattern for 3
    assert call(2, [(0, 0), (128, 0)]) == B.LR_ERR_INVALID_ARG
    assert call(4, None, nb=W * H * 16 * 4) == B.LR_ERR_OOM  # room for the images only
    torch.cuda.synchronize()
