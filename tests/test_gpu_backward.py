"""Backward pass of the compositing w.r.t. flat per-quad RGBA, checked against the fp64
CPU oracle gradient (1e-3 relative) and against the GPU forward's own central differences.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from scenegen import COLOR_FLAT

pytestmark = pytest.mark.gpu


def _rel_ok(g, ref, rtol=1e-3):
    scale = 1e-3 * np.abs(ref).max()
    err = np.abs(g - ref)
    return np.all(err <= rtol * np.maximum(np.abs(ref), scale)), err.max()


@pytest.mark.parametrize("k", [1, 3])
def test_backward_matches_fp64_oracle(k):
    import paper_2405_13364_gb300 as P
    s = scenegen.wavy_layers(160, 128, layers=16, nx=24, ny=24, seed=4, color_mode=COLOR_FLAT,
                             half_h=2.0, dz=0.3)
    target = oracle.render(s.with_colors(scenegen.perturbed_target_colors(s.colors, seed=1)))["rgba"]
    r = P.Renderer(sorter_k=k)
    ds = P.DeviceScene.from_scene(s)
    colors = torch.tensor(s.colors, device="cuda", requires_grad=True)
    img = P.composite(colors, r, ds, s.width, s.height)
    tgt = torch.tensor(target, device="cuda")
    loss = ((img[..., :3] - tgt[..., :3]) ** 2).sum()
    loss.backward()
    g = colors.grad.cpu().numpy().astype(np.float64)
    col64 = s.colors.astype(np.float64)
    ref = oracle.backward(s, oracle.loss_l2_grad(oracle.render64(s, col64), target), col64)
    ok, worst = _rel_ok(g, ref)
    assert ok, worst
    rel_l2 = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel_l2 < 1e-3
    r.close()


def test_backward_one_layer_closed_form():
    import paper_2405_13364_gb300 as P
    from tests.scene_helpers import rects_scene
    c = np.array([[0.3, 0.6, 0.9, 0.4]], np.float32)
    s = rects_scene([(2.0, 2.0, 6.0, 5.0)], colors=c)
    r = P.Renderer()
    colors = torch.tensor(c, device="cuda", requires_grad=True)
    img = P.composite(colors, r, P.DeviceScene.from_scene(s), 16, 16)
    (img[..., :3] ** 2).sum().backward()
    g = colors.grad.cpu().numpy()[0]
    a, col = 0.4, c[0, :3].astype(np.float64)
    np.testing.assert_allclose(g[:3], 12 * 2 * (a * col) * a, rtol=1e-5)
    np.testing.assert_allclose(g[3], 12 * np.sum(2 * (a * col) * col), rtol=1e-5)
    r.close()
