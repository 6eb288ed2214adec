"""The alpha-threshold and lit modes through the other entry points: captured CUDA graphs
(replays keep the light they were captured with), the serving loop (its context's light),
and HostStream (32-byte lit vertex colours copied from pinned host memory)."""
import dataclasses
import time

import numpy as np
import pytest
import torch

import oracle
import scenegen
from scenegen import COLOR_LIT

pytestmark = pytest.mark.gpu

COLOR_TOL = 1e-5


def _close(a, b, tol):
    return float(np.abs(a.astype(np.float64) - b.astype(np.float64)).max()) <= tol


def test_threshold_graph_replay_equals_direct():
    import paper_2405_13364_gb300 as P
    scenes = [scenegen.wavy_layers(256, 144, layers=24, nx=24, ny=12, seed=1),
              scenegen.gaussian_particles(30_000, 256, 144, seed=2)]
    r = P.Renderer(sorter_k=3, alpha_threshold=True)
    items = [(P.DeviceScene.from_scene(s), s.width, s.height) for s in scenes]
    g = r.capture(items)
    for _ in range(2):
        outs = g.launch()
    torch.cuda.synchronize()
    for (d, w, h), o in zip(items, outs):
        direct = r.render(d, w, h)["rgba"]
        torch.cuda.synchronize()
        assert torch.equal(o["rgba"], direct)
    g.close()
    r.close()


def test_lit_graph_replay_keeps_captured_light():
    import paper_2405_13364_gb300 as P
    s = scenegen.wavy_layers(200, 120, layers=16, nx=20, ny=12, seed=3, color_mode=COLOR_LIT)
    d = P.DeviceScene.from_scene(s)
    r = P.Renderer(sorter_k=3)
    r.set_lighting(s.light[:3], s.light[3])
    g = r.capture([(d, s.width, s.height)])
    ref_a = r.render(d, s.width, s.height)["rgba"]
    r.set_lighting((0.0, -1.0, 0.2), 0.1)             # later renders use the new light
    out = g.launch([(d, s.width, s.height)])[0]["rgba"]
    ref_b = r.render(d, s.width, s.height)["rgba"]
    torch.cuda.synchronize()
    assert torch.equal(out, ref_a)
    assert not torch.equal(out, ref_b)
    assert _close(ref_a.cpu().numpy(), oracle.render(s)["rgba"], COLOR_TOL)
    g.close()
    r.close()


def test_lit_requests_served_with_the_servers_light():
    import paper_2405_13364_gb300 as P
    light = (0.3, 0.8, 0.6, 0.2)
    scenes = []
    for i in range(8):
        w, h = [(192, 128), (160, 96)][i % 2]
        mode = COLOR_LIT if i % 2 == 0 else scenegen.COLOR_VERTEX
        s = scenegen.wavy_layers(w, h, layers=12, nx=16, ny=8, seed=i, color_mode=mode)
        if mode == COLOR_LIT:
            s = dataclasses.replace(s, light=light)
        scenes.append(s)
    ds = [P.DeviceScene.from_scene(s) for s in scenes]
    srv = P.Server(sorter_k=3, num_slots=2, max_batch_views=4, slot_workspace_bytes=128 << 20, light=light)
    tickets = [srv.submit(d, s.width, s.height) for s, d in zip(scenes, ds)]
    results = {}
    deadline = time.time() + 60
    while len(results) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in results:
                r = srv.poll(t, timeout_us=1000)
                if r is not None:
                    results[t] = r
    assert len(results) == len(tickets)
    torch.cuda.synchronize()
    for t, s in zip(tickets, scenes):
        status, out, _ = results[t]
        assert status == 0
        assert _close(out["rgba"].cpu().numpy(), oracle.render(s)["rgba"], COLOR_TOL)


def test_host_stream_lit_colours():
    import paper_2405_13364_gb300 as P
    s = scenegen.wavy_layers(160, 96, layers=12, nx=16, ny=10, seed=11, color_mode=COLOR_LIT)
    r = P.Renderer(sorter_k=3)
    r.set_lighting(s.light[:3], s.light[3])
    hs = P.HostStream(r, s.positions.shape[0], s.num_quads, True, s.color_mode, s.colors.shape[0],
                      s.width, s.height)
    out = torch.empty((s.height, s.width, 4), dtype=torch.float32).pin_memory()
    pos = torch.from_numpy(s.positions).pin_memory()
    idx = torch.from_numpy(s.indices.view(np.int32)).pin_memory()
    col = torch.from_numpy(s.colors).pin_memory()
    for _ in range(2):
        hs.submit(pos, idx, col, s.view_proj, s.near, s.far, out)
    hs.synchronize()
    ref = r.render(P.DeviceScene.from_scene(s), s.width, s.height)["rgba"]
    torch.cuda.synchronize()
    assert torch.equal(out, ref.cpu())
    assert _close(out.numpy(), oracle.render(s)["rgba"], COLOR_TOL)
    r.close()
