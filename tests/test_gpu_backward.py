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


@pytest.mark.parametrize("k", [1, 2])
def test_backward_with_forward_mask(k):
    # the forward's exact-path mask lets the backward skip its detection pass: same
    # gradients (up to the order of fp32 atomics) and the same flagged pixels; a mask that
    # misses flagged pixels is reported (LR_ERR_MASK_MISMATCH), and render_backward then
    # repeats the call without it
    import paper_2405_13364_gb300 as P
    from paper_2405_13364_gb300 import _binding as B
    s = scenegen.wavy_layers(200, 136, layers=20, nx=24, ny=20, seed=7, color_mode=COLOR_FLAT,
                             half_h=2.0, dz=0.25)
    r = P.Renderer(sorter_k=k)
    ds = P.DeviceScene.from_scene(s)
    fwd = r.render(ds, s.width, s.height, exact_mask=True)
    torch.cuda.synchronize()
    flagged = int(r.stats()["overflow_pixels"])
    mask = fwd["exact_mask"]
    bits = int(sum(bin(int(w) & 0xFFFFFFFF).count("1") for w in mask.flatten().tolist()))
    assert bits == flagged
    if k == 1:
        assert flagged > 0
    g_out = torch.randn_like(fwd["rgba"])
    g0 = r.render_backward(ds, s.width, s.height, fwd["rgba"], g_out)
    g1 = r.render_backward(ds, s.width, s.height, fwd["rgba"], g_out, exact_mask=mask)
    torch.cuda.synchronize()
    assert int(r.stats()["overflow_pixels"]) == flagged
    scale = float(g0.abs().max())
    assert float((g0 - g1).abs().max()) <= 1e-5 * scale
    if flagged == 0:
        r.close()
        return
    # a mask that misses the flagged pixels: detected on the GPU, reported on the host
    zero = torch.zeros_like(mask)
    grad = torch.zeros((s.num_quads, 4), dtype=torch.float32, device="cuda")
    view = r.view_struct(ds, s.width, s.height, P.Outputs(rgba=fwd["rgba"]))
    ptr, nbytes = r.workspace(B.lr_workspace_size_batch(r.ctx, [view]))
    B.lr_render_backward(r.ctx, ds.quads_struct(), ds.camera_struct(), s.width, s.height,
                         fwd["rgba"].data_ptr(), g_out.data_ptr(), zero.data_ptr(), grad.data_ptr(),
                         ptr, nbytes, torch.cuda.current_stream().cuda_stream)
    st = B.lr_get_stats(r.ctx, raise_on_error=False)
    assert st.status == B.LR_ERR_MASK_MISMATCH
    g2 = r.render_backward(ds, s.width, s.height, fwd["rgba"], g_out, exact_mask=zero)
    torch.cuda.synchronize()
    assert float((g0 - g2).abs().max()) <= 1e-5 * scale
    r.close()
