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


def test_served_mixed_resolutions_match_oracle():
    # requests at every served resolution up to 2560x1440, each with its own sorter
    # capacity: served = rendered alone (bitwise), and a subset against the oracle
    import oracle
    import paper_2405_13364_gb300 as P
    reqs = []
    for i, (w, h) in enumerate([(1920, 1080), (2560, 1440), (256, 256), (1024, 768), (1920, 1080),
                                (2560, 1440), (1024, 768), (1920, 1080)]):
        kind = ("particles", "layers", "frustum")[i % 3]
        q = (200_000, 120_000, 20_000, 60_000, 150_000, 40_000, 90_000, 400_000)[i]
        reqs.append((scenegen.scene_for_request(dict(kind=kind, quads=q, width=w, height=h, seed=50 + i)),
                     (1, 2, 3)[i % 3]))
    srv = P.Server(sorter_k=3, num_slots=2, max_batch_views=4, slot_workspace_bytes=1 << 30)
    dev = [P.DeviceScene.from_scene(s) for s, _ in reqs]
    tickets = [srv.submit(d, s.width, s.height, count=True, hash=True, sorter_k=k)
               for d, (s, k) in zip(dev, reqs)]
    results = []
    for t in tickets:
        r = None
        deadline = time.time() + 60
        while r is None and time.time() < deadline:
            r = srv.poll(t, timeout_us=100_000)
        assert r is not None and r[0] == 0
        results.append(r[1])
    torch.cuda.synchronize()
    srv.close()
    alone = P.Renderer(sorter_k=3)
    for (s, k), d, out in zip(reqs, dev, results):
        ref = alone.make_outputs(s.width, s.height, count=True, hash=True)
        alone.render_views([alone.view_struct(d, s.width, s.height, ref, sorter_k=k)])
        torch.cuda.synchronize()
        assert torch.equal(out["rgba"], ref["rgba"]) and torch.equal(out["count"], ref["count"])
        assert torch.equal(out["hash"], ref["hash"])
    alone.close()
    # the oracle on the requests up to 1920x1080 x 200k quads, and one at 2560x1440
    for i in (0, 2, 3, 4, 5):
        s, _ = reqs[i]
        o = oracle.render(s)
        out = results[i]
        np.testing.assert_array_equal(out["count"].cpu().numpy().view(np.uint32), o["count"])
        np.testing.assert_array_equal(out["hash"].cpu().numpy().view(np.uint64), o["hash"])
        d = np.abs(out["rgba"].cpu().numpy().astype(np.float64) - o["rgba"]).max()
        assert d <= 1e-5, (i, d)


def test_batch_with_per_view_sorter_capacity():
    # a batch whose views ask for another capacity equals a context of that capacity;
    # mixed capacities in one batch are refused
    import paper_2405_13364_gb300 as P
    from paper_2405_13364_gb300 import _binding as B
    s = scenegen.wavy_layers(200, 120, layers=16, nx=20, ny=10, seed=4)
    d = P.DeviceScene.from_scene(s)
    r3 = P.Renderer(sorter_k=3)
    o1 = r3.make_outputs(s.width, s.height, count=True)
    st = r3.render_views([r3.view_struct(d, s.width, s.height, o1, sorter_k=1)])
    torch.cuda.synchronize()
    r1 = P.Renderer(sorter_k=1)
    ref = r1.render(d, s.width, s.height, count=True)
    st1 = r1.stats()
    torch.cuda.synchronize()
    assert torch.equal(o1["rgba"], ref["rgba"]) and torch.equal(o1["count"], ref["count"])
    assert st.overflow_pixels == st1["overflow_pixels"] > 0     # K = 1 really ran
    o2 = r3.make_outputs(s.width, s.height)
    views = [r3.view_struct(d, s.width, s.height, o1, sorter_k=1), r3.view_struct(d, s.width, s.height, o2, sorter_k=2)]
    with pytest.raises(P.LrError) as e:
        r3.render_views(views)
    assert e.value.status == B.LR_ERR_INVALID_ARG
    with pytest.raises(P.LrError):
        r3.render_views([r3.view_struct(d, s.width, s.height, o2, sorter_k=5)])
    r1.close()
    r3.close()
