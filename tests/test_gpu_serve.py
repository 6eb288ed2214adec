"""Serving (continuous batching): every served result equals the same request rendered
alone (bitwise: the pipeline is exact and deterministic), requests are batched, and the
server drains cleanly."""
import time

import numpy as np
import pytest
import torch

import scenegen

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    for i in range(24):
        kind = i % 3
        w, h = [(256, 256), (320, 200), (200, 120)][i % 3]
        if kind == 0:
            s = scenegen.frustum_parallelograms(1500 + 100 * i, w, h, seed=i)
        elif kind == 1:
            s = scenegen.wavy_layers(w, h, layers=12, nx=16, ny=8, seed=i)
        else:
            s = scenegen.gaussian_particles(8000 + 500 * i, w, h, seed=i)
        out.append(s)
    return out


def test_served_equals_alone():
    import paper_2405_13364_gb300 as P
    scenes = _requests()
    dscenes = [P.DeviceScene.from_scene(s) for s in scenes]
    alone = P.Renderer(sorter_k=3)
    ref = []
    for s, d in zip(scenes, dscenes):
        o = alone.render(d, s.width, s.height, count=True)
        ref.append((o["rgba"].cpu().numpy(), o["count"].cpu().numpy()))
    alone.close()
    srv = P.Server(sorter_k=3, num_slots=2, max_batch_views=8, slot_workspace_bytes=256 << 20)
    tickets = [srv.submit(d, s.width, s.height, count=True) for s, d in zip(scenes, dscenes)]
    results = {}
    deadline = time.time() + 60
    while len(results) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t in results:
                continue
            r = srv.poll(t, timeout_us=1000)
            if r is not None:
                results[t] = r
    assert len(results) == len(tickets)
    for t, (rgba_ref, cnt_ref) in zip(tickets, ref):
        status, out, info = results[t]
        assert status == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out["rgba"].cpu().numpy(), rgba_ref)
        np.testing.assert_array_equal(out["count"].cpu().numpy(), cnt_ref)
        assert info["done_ns"] >= info["launch_ns"] >= info["submit_ns"]
    st = srv.stats()
    assert st["completed"] == len(tickets) and st["failed"] == 0
    assert st["batches"] < len(tickets)     # requests were batched
    srv.close()


def test_oversized_request_rejected_others_served():
    import paper_2405_13364_gb300 as P
    small = scenegen.frustum_parallelograms(500, 64, 64, seed=1)
    big = scenegen.gaussian_particles(400_000, 1920, 1080, seed=2)
    srv = P.Server(sorter_k=3, num_slots=1, max_batch_views=4, slot_workspace_bytes=16 << 20)
    t_big = srv.submit(P.DeviceScene.from_scene(big), 1920, 1080)
    t_small = srv.submit(P.DeviceScene.from_scene(small), 64, 64)
    rb = srv.poll(t_big, timeout_us=5_000_000)
    rs = srv.poll(t_small, timeout_us=5_000_000)
    assert rb is not None and rb[0] == -3          # LR_ERR_OOM: does not fit a slot
    assert rs is not None and rs[0] == 0
    srv.close()
