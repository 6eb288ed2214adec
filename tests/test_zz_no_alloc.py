"""lr_render_noalloc: the render entry point for callers that cannot allocate device
memory when they render (e.g. a per-frame plugin whose host application owns all device
memory and forbids cudaMalloc after start-up). It renders on a scratch array built into
the library instead of a caller workspace.

Checked through the C ABI against the existing lr_render entry point (same pipeline,
K = 3) on two calls in a row, within the colour tolerance of the other parity tests.
This file is collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest
import torch

import scenegen

pytestmark = pytest.mark.gpu

COLOR_TOL = 1e-5


def _scenes():
    return [scenegen.config_small_frustum(),
            scenegen.wavy_layers(333, 190, layers=32, nx=48, ny=24, seed=1)]


@pytest.mark.parametrize("k", [0, 1])
def test_noalloc_matches_lr_render_twice(k):
    import paper_2405_13364_gb300 as P
    from paper_2405_13364_gb300 import _binding as B
    scene = _scenes()[k]
    W, H = scene.width, scene.height
    r = P.Renderer(sorter_k=3)
    ds = P.DeviceScene.from_scene(scene)
    # existing entry point, through the C ABI
    ref = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    need = B.lr_workspace_size(r.ctx, ds.num_quads, W, H)
    ptr, nbytes = r.workspace(need)
    stream = torch.cuda.current_stream()
    B.lr_render(r.ctx, ds.quads_struct(), ds.camera_struct(), W, H, int(ref.data_ptr()), ptr, nbytes,
                stream.cuda_stream)
    assert B.lr_get_stats(r.ctx).status == 0
    ref_np = ref.cpu().numpy()
    # the allocation-free entry point, two calls in a row into fresh outputs; the device's
    # free memory (what cudaMemGetInfo reports) must not move across the second call
    status = torch.empty((1,), dtype=torch.int32, device="cuda")
    for call in range(2):
        out = torch.full((H, W, 4), float("nan"), dtype=torch.float32, device="cuda")
        status.fill_(12345)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = B.lr_render_noalloc(ds.quads_struct(), ds.camera_struct(), W, H, int(out.data_ptr()),
                                 int(status.data_ptr()), stream.cuda_stream)
        assert rc == B.LR_OK, (call, rc)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert int(status.item()) == B.LR_OK
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        err = np.abs(got.astype(np.float64) - ref_np.astype(np.float64)).max()
        assert err <= COLOR_TOL, (call, err)
    r.close()


def test_noalloc_rejects_scenes_beyond_its_scratch():
    import paper_2405_13364_gb300 as P
    from paper_2405_13364_gb300 import _binding as B
    scene = scenegen.config_small_frustum()
    ds = P.DeviceScene.from_scene(scene)
    q = ds.quads_struct()
    q.num_quads = 4_000_000          # far more than the scratch array holds; nothing is read
    out = torch.zeros((64, 64, 4), dtype=torch.float32, device="cuda")
    rc = B.lr_render_noalloc(q, ds.camera_struct(), 64, 64, int(out.data_ptr()), None,
                             torch.cuda.current_stream().cuda_stream)
    assert rc == B.LR_ERR_TOO_LARGE
    rc = B.lr_render_noalloc(ds.quads_struct(), ds.camera_struct(), 20000, 20000, int(out.data_ptr()),
                             None, torch.cuda.current_stream().cuda_stream)
    assert rc == B.LR_ERR_TOO_LARGE
    torch.cuda.synchronize()


def test_noalloc_reports_reference_overflow():
    # 2,000 screen-filling quads at 1920x1080 pass the host-side check (two references per
    # quad) but need 2,040 references each, far more than the array holds: the GPU status
    # word says so and the image is left as it was
    import paper_2405_13364_gb300 as P
    from paper_2405_13364_gb300 import _binding as B
    from tests.scene_helpers import rects_scene
    W, H = 1920, 1080
    rects = [(0.25, 0.25, W - 0.25, H - 0.25)] * 2000
    s = rects_scene(rects, width=W, height=H)
    ds = P.DeviceScene.from_scene(s)
    out = torch.full((H, W, 4), float("nan"), dtype=torch.float32, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    rc = B.lr_render_noalloc(ds.quads_struct(), ds.camera_struct(), W, H, int(out.data_ptr()),
                             int(status.data_ptr()), torch.cuda.current_stream().cuda_stream)
    assert rc == B.LR_OK
    torch.cuda.synchronize()
    assert int(status.item()) == B.LR_ERR_OVERFLOW
    assert bool(torch.isnan(out).all())
