"""HostStream: frames rendered from host memory with the copies of neighbouring frames
overlapping rendering equal, bit for bit, the same frames rendered one at a time from
device memory, and match the oracle."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from tests.test_gpu_parity import assert_parity, gpu_render

pytestmark = pytest.mark.gpu


def test_host_stream_matches_device_renders():
    import paper_2405_13364_gb300 as P
    P.load_library()
    base = scenegen.wavy_layers(160, 96, layers=12, nx=16, ny=10, seed=11)
    rng = np.random.default_rng(5)
    frames = []
    for i in range(5):
        col = np.clip(base.colors * rng.uniform(0.5, 1.0, (1, 4)).astype(np.float32), 0, 1).astype(np.float32)
        frames.append(scenegen.Scene(base.positions, base.indices, col, base.color_mode, base.view_proj,
                                     base.near, base.far, base.width, base.height))
    r = P.Renderer(sorter_k=3)
    hs = P.HostStream(r, base.positions.shape[0], base.num_quads, True, base.color_mode, base.colors.shape[0],
                      base.width, base.height)
    outs = [torch.empty((base.height, base.width, 4), dtype=torch.float32).pin_memory() for _ in frames]
    pos = torch.from_numpy(base.positions).pin_memory()
    idx = torch.from_numpy(base.indices.view(np.int32)).pin_memory()
    for s, o in zip(frames, outs):
        hs.submit(pos, idx, torch.from_numpy(s.colors).pin_memory(), s.view_proj, s.near, s.far, o)
    hs.synchronize()
    for s, o in zip(frames, outs):
        ref = r.render(P.DeviceScene.from_scene(s), s.width, s.height)
        torch.cuda.synchronize()
        assert torch.equal(o, ref["rgba"].cpu())
    g = gpu_render(P, frames[-1])
    g["rgba"] = outs[-1].numpy()
    assert_parity(g, oracle.render(frames[-1]))
    r.close()
