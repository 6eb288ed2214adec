"""GPU parity of the lit colour mode (LR_COLOR_LIT: per-vertex colours and normals, one
directional light, two-sided Lambert plus ambient) with the oracle. Bar: linear fp32 RGBA
within 1e-5 of the oracle per channel; coverage and order are the exact integer work of
the other modes and are unaffected. Every call goes through the C ABI via the ctypes
binding."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import scenegen
from scenegen import COLOR_LIT

pytestmark = pytest.mark.gpu

COLOR_TOL = 1e-5


@pytest.fixture(scope="module")
def lr():
    import paper_2405_13364_gb300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    P.load_library()
    return P


def lit_renderer(lr, scene, k=3, **kw):
    r = lr.Renderer(sorter_k=k, **kw)
    r.set_lighting(scene.light[:3], scene.light[3])
    return r


def lit_layers(w=333, h=190, seed=1, light=None):
    s = scenegen.wavy_layers(w, h, layers=32, nx=48, ny=24, seed=seed, color_mode=COLOR_LIT)
    return s if light is None else dataclasses.replace(s, light=light)


def assert_close(g, o, tol=COLOR_TOL):
    d = np.abs(g.astype(np.float64) - o.astype(np.float64))
    assert d.max() <= tol, f"max colour error {d.max()} at {np.unravel_index(d.argmax(), d.shape)}"


@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("light", [None, (-0.7, 0.2, 0.4, 0.0), (0.0, 0.0, -1.0, 0.6)])
def test_lit_matches_oracle(lr, k, light):
    scene = lit_layers(light=light)
    r = lit_renderer(lr, scene, k)
    out = r.render(lr.DeviceScene.from_scene(scene), scene.width, scene.height, count=True)
    torch.cuda.synchronize()
    o = oracle.render(scene)
    np.testing.assert_array_equal(out["count"].cpu().numpy().view(np.uint32), o["count"])
    assert_close(out["rgba"].cpu().numpy(), o["rgba"])
    r.close()


def test_mixed_batch_lit_vertex_flat(lr):
    lit = lit_layers(200, 150, seed=2)
    vtx = scenegen.wavy_layers(180, 120, layers=24, nx=24, ny=16, seed=3)
    flat = scenegen.gaussian_particles(20_000, 160, 96, seed=4)
    r = lit_renderer(lr, lit, 3)
    items = [(lr.DeviceScene.from_scene(s), s.width, s.height) for s in (lit, vtx, flat)]
    outs = r.render_batch(items)
    torch.cuda.synchronize()
    for s, o in zip((lit, vtx, flat), outs):
        assert_close(o["rgba"].cpu().numpy(), oracle.render(s)["rgba"])
    r.close()


def test_lit_msaa(lr):
    scene = lit_layers(160, 96, seed=5)
    r = lit_renderer(lr, scene, 3)
    out = r.render_msaa(lr.DeviceScene.from_scene(scene), scene.width, scene.height, samples=4)
    torch.cuda.synchronize()
    want, _ = oracle.render_msaa(scene, 4)
    assert_close(out.cpu().numpy(), want)
    r.close()


def test_lit_full_size_layers(lr):
    # the 1920x1080 layer frame (1M quads) with lit colours, K = 1 (exact path exercised)
    scene = scenegen.wavy_layers(color_mode=COLOR_LIT)
    r = lit_renderer(lr, scene, 1)
    out = r.render(lr.DeviceScene.from_scene(scene), scene.width, scene.height)
    torch.cuda.synchronize()
    st = r.stats()
    assert st["overflow_pixels"] > 0
    assert_close(out["rgba"].cpu().numpy(), oracle.render(scene)["rgba"])
    r.close()


def test_lit_refusals(lr):
    from paper_2405_13364_gb300 import _binding as B
    scene = lit_layers(64, 48)
    r = lit_renderer(lr, scene, 3)
    ds = lr.DeviceScene.from_scene(scene)
    with pytest.raises(B.LrError) as e:
        r.render(ds, scene.width, scene.height, hash=True)
    assert e.value.status == B.LR_ERR_UNSUPPORTED
    with pytest.raises(B.LrError) as e:
        r.set_lighting((0.0, 0.0, 0.0), 0.2)
    assert e.value.status == B.LR_ERR_INVALID_ARG
    with pytest.raises(B.LrError) as e:
        r.set_lighting((0.0, 1.0, 0.0), 1.5)
    assert e.value.status == B.LR_ERR_INVALID_ARG
    rt = lit_renderer(lr, scene, 3, alpha_threshold=True)
    with pytest.raises(B.LrError) as e:
        rt.render(ds, scene.width, scene.height)
    assert e.value.status == B.LR_ERR_UNSUPPORTED
    with pytest.raises(B.LrError) as e:
        r.render_backward(ds, scene.width, scene.height,
                          torch.zeros((scene.height, scene.width, 4), device="cuda"),
                          torch.zeros((scene.height, scene.width, 4), device="cuda"))
    assert e.value.status == B.LR_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    r.close()
    rt.close()
