"""Differentiable compositing at full size: 1024x1024, 524,288 quads (layer generator,
flat RGBA), L = squared L2 distance to a target rendered with RGBA + N(0, 0.05) clamped.
The GPU gradient (lr_render_backward through torch.autograd) must be within 1e-3
relative of the fp64 oracle gradient; central differences of the GPU forward (h = 1e-3)
on 64 random quads x 4 channels are checked against it as well.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen

pytestmark = pytest.mark.gpu


def test_full_size_gradient():
    import paper_2405_13364_gb300 as P
    s = scenegen.config_diff_1024()
    tcol = scenegen.perturbed_target_colors(s.colors, seed=1)
    target = oracle.render(s.with_colors(tcol))["rgba"]
    r = P.Renderer(sorter_k=3)
    ds = P.DeviceScene.from_scene(s)
    colors = torch.tensor(s.colors, device="cuda", requires_grad=True)
    tgt = torch.tensor(target, device="cuda")
    img = P.composite(colors, r, ds, s.width, s.height)
    loss = ((img[..., :3] - tgt[..., :3]) ** 2).sum()
    loss.backward()
    g = colors.grad.cpu().numpy().astype(np.float64)

    col64 = s.colors.astype(np.float64)
    ref = oracle.backward(s, oracle.loss_l2_grad(oracle.render64(s, col64), target), col64)
    scale = 1e-3 * np.abs(ref).max()
    err = np.abs(g - ref)
    assert np.all(err <= 1e-3 * np.maximum(np.abs(ref), scale)), float((err / np.maximum(np.abs(ref), scale)).max())
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-3

    # central differences of the GPU forward on 64 random quads; a colour only changes the
    # pixels in its quad's box, so the loss difference is summed there (in fp64)
    st = oracle.setup(s)
    vis = np.nonzero(st["status"] == 0)[0]
    rng = np.random.default_rng(2)
    picks = rng.choice(vis, 64, replace=False)
    h = 1e-3
    t_np = target[..., :3].astype(np.float64)
    fd, an = [], []
    base = colors.detach().clone()
    for j in picks:
        x0, x1, y0, y1 = st["bbox"][j]
        for ch in range(4):
            vals = []
            for sgn in (1.0, -1.0):
                c = base.clone()
                c[j, ch] += sgn * h
                im = r.render(ds.with_colors(c), s.width, s.height)["rgba"]
                reg = im[y0:y1 + 1, x0:x1 + 1, :3].double().cpu().numpy()
                vals.append(((reg - t_np[y0:y1 + 1, x0:x1 + 1]) ** 2).sum())
            fd.append((vals[0] - vals[1]) / (2 * h))
            an.append(g[j, ch])
    fd, an = np.array(fd), np.array(an)
    rel = np.linalg.norm(fd - an) / np.linalg.norm(an)
    print(f"GPU-forward central differences vs GPU gradient: relative L2 error {rel:.2e}")
    assert rel < 5e-3
    r.close()
