"""Batched multi-view launches and captured CUDA graphs give the same images as single
renders; graph replays can swap scenes and cameras of the same shape."""
import numpy as np
import pytest
import torch

import oracle
import scenegen

pytestmark = pytest.mark.gpu


def _scenes():
    return [scenegen.wavy_layers(256, 144, layers=12, nx=24, ny=12, seed=1),
            scenegen.gaussian_particles(20_000, 256, 144, seed=2),
            scenegen.frustum_parallelograms(3000, 256, 144, seed=3)]


def test_graph_replay_matches_oracle_and_swaps_scenes():
    import paper_2405_13364_gb300 as P
    scenes = _scenes()
    r = P.Renderer(sorter_k=3)
    items = [(P.DeviceScene.from_scene(s), s.width, s.height) for s in scenes]
    g = r.capture(items, count=True)
    outs = g.launch()
    torch.cuda.synchronize()
    for s, o in zip(scenes, outs):
        ref = oracle.render(s)
        np.testing.assert_array_equal(o["count"].cpu().numpy().view(np.uint32), ref["count"])
        assert np.abs(o["rgba"].cpu().numpy().astype(np.float64) - ref["rgba"]).max() <= 1e-5
    # swap in other scenes of the same shape (same quad counts, resolution, colour mode)
    scenes2 = [scenegen.wavy_layers(256, 144, layers=12, nx=24, ny=12, seed=7),
               scenegen.gaussian_particles(20_000, 256, 144, seed=8),
               scenegen.frustum_parallelograms(3000, 256, 144, seed=9)]
    items2 = [(P.DeviceScene.from_scene(s), s.width, s.height) for s in scenes2]
    for _ in range(3):
        outs = g.launch(items2)
    torch.cuda.synchronize()
    for s, o in zip(scenes2, outs):
        ref = oracle.render(s)
        np.testing.assert_array_equal(o["count"].cpu().numpy().view(np.uint32), ref["count"])
        assert np.abs(o["rgba"].cpu().numpy().astype(np.float64) - ref["rgba"]).max() <= 1e-5
    g.close()
    r.close()


def test_graph_rejects_shape_change():
    import paper_2405_13364_gb300 as P
    s = _scenes()[1]
    r = P.Renderer()
    g = r.capture([(P.DeviceScene.from_scene(s), s.width, s.height)])
    other = scenegen.gaussian_particles(10_000, 256, 144, seed=2)
    with pytest.raises(P.LrError):
        g.launch([(P.DeviceScene.from_scene(other), 256, 144)])
    g.close()
    r.close()
