"""Full-size parity of the exact path with the oracle on the two 1920x1080 workloads
(stacked layers: 1,048,576 indexed quads with per-vertex colours; particles: 2,000,000
flat-colour squares with depth complexity above 1,000), on the rasteriser instances the
benchmark times, and on the sort branches of the dense-bin path.

Bar (as everywhere): per-pixel fragment counts and coverage hashes bit-exact, linear fp32
RGBA within 1e-5 per channel, 8-bit output within 1 LSB, the fragment total equal to the
oracle's. Every call goes through the C ABI.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from tests.scene_helpers import rects_scene

pytestmark = pytest.mark.gpu

COLOR_TOL = 1e-5

_oracle_cache = {}


def _scene(name):
    return {"layers": scenegen.config_layers_1080p, "particles": scenegen.config_particles_1080p}[name]()


def _oracle(name):
    if name not in _oracle_cache:
        s = _scene(name)
        _oracle_cache[name] = (s, oracle.render(s))
    return _oracle_cache[name]


@pytest.fixture(scope="module")
def lr():
    import paper_2405_13364_gb300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    P.load_library()
    return P


def _compare(out, st, o, counts=True, hashes=False):
    rgba = out["rgba"].cpu().numpy()
    d = np.abs(rgba.astype(np.float64) - o["rgba"].astype(np.float64))
    assert d.max() <= COLOR_TOL, f"max colour error {d.max()} at {np.unravel_index(d.argmax(), d.shape)}"
    if "rgba8" in out:
        d8 = np.abs(out["rgba8"].cpu().numpy().astype(np.int32) - o["rgba8"].astype(np.int32))
        assert d8.max() <= 1
    if counts:
        np.testing.assert_array_equal(out["count"].cpu().numpy().view(np.uint32), o["count"])
    if hashes:
        np.testing.assert_array_equal(out["hash"].cpu().numpy().view(np.uint64), o["hash"])
    assert st["fragments"] == int(o["count"].sum()) == o["stats"]["fragments"]
    assert st["quads_visible"] == o["stats"]["visible"]


@pytest.mark.parametrize("name", ["layers", "particles"])
@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("carry", [False, True])
def test_full_size_benched_instance(lr, name, k, carry):
    # the rasteriser instance the benchmark launches (no coverage hash), with counts and the
    # 8-bit image written beside the colour; carry only matters for flat colours
    if carry and name == "layers":
        pytest.skip("per-vertex colours are always carried")
    s, o = _oracle(name)
    r = lr.Renderer(sorter_k=k, carry_colors=carry)
    out = r.render(lr.DeviceScene.from_scene(s), s.width, s.height, rgba8=True, count=True)
    torch.cuda.synchronize()
    st = r.stats()
    assert st["status"] == 0
    _compare(out, st, o)
    if k == 1 and name == "layers":
        assert st["overflow_pixels"] > 0      # interpenetrating layers: the exact path ran
    if name == "particles":
        assert st["bins_high"] > 0 and sum(st["sort_bins"]) == st["bins_high"]
    r.close()


@pytest.mark.parametrize("name", ["layers", "particles"])
def test_full_size_image_only(lr, name):
    # exactly the benchmark's call: the colour image alone, autotuned-size sorter (K = 1)
    s, o = _oracle(name)
    r = lr.Renderer(sorter_k=1)
    out = r.render(lr.DeviceScene.from_scene(s), s.width, s.height)
    torch.cuda.synchronize()
    _compare(out, r.stats(), o, counts=False)
    r.close()


@pytest.mark.parametrize("name", ["layers", "particles"])
def test_full_size_hashes(lr, name):
    s, o = _oracle(name)
    r = lr.Renderer(sorter_k=1)
    out = r.render(lr.DeviceScene.from_scene(s), s.width, s.height, rgba8=True, count=True, hash=True)
    torch.cuda.synchronize()
    _compare(out, r.stats(), o, hashes=True)
    r.close()


def _particles_in_one_bin(n, seed):
    # a 32 x 32 image is one bin; squares of 2-4 px at Gaussian depths (distinct keys)
    return scenegen.gaussian_particles(n, 32, 32, seed=seed, sigma=1.5, size_px=(2.0, 4.0))


def _render_counted(lr, s, k=3):
    r = lr.Renderer(sorter_k=k)
    out = r.render(lr.DeviceScene.from_scene(s), s.width, s.height, rgba8=True, count=True, hash=True)
    torch.cuda.synchronize()
    st = r.stats()
    r.close()
    return out, st


def test_sort_branch_global_merge(lr):
    # more than 20480 references in one bin, distinct depths: runs of 8192 sorted in shared
    # memory and merged through global memory
    s = _particles_in_one_bin(30_000, seed=21)
    out, st = _render_counted(lr, s)
    assert st["max_bin_refs"] > 20480
    assert st["sort_bins"][2] == 1 and st["bins_high"] == 1
    _compare(out, st, oracle.render(s), hashes=True)


def test_sort_branch_bucket(lr):
    # 2048..20480 references with distinct depths: the bucket sort
    s = _particles_in_one_bin(6_000, seed=22)
    out, st = _render_counted(lr, s)
    assert 2048 <= st["max_bin_refs"] <= 20480
    assert st["sort_bins"][0] == 1
    _compare(out, st, oracle.render(s), hashes=True)


def test_sort_branch_shared_merge(lr):
    # 2048..8192 references all at one depth: every key in one bucket, so the bucket sort
    # gives up and the merge sort runs in shared memory alone
    rng = np.random.default_rng(23)
    rects = []
    for _ in range(4000):
        x0, y0 = rng.uniform(0, 24, 2)
        rects.append((float(np.floor(x0 * 4) / 4), float(np.floor(y0 * 4) / 4),
                      float(np.floor(x0 * 4) / 4 + 6.0), float(np.floor(y0 * 4) / 4 + 5.0)))
    cols = np.concatenate([rng.random((4000, 3)), rng.uniform(0.02, 0.2, (4000, 1))], 1)
    s = rects_scene(rects, width=32, height=32, colors=cols)
    out, st = _render_counted(lr, s)
    assert 2048 <= st["max_bin_refs"] <= 8192
    assert st["sort_bins"][1] == 1
    _compare(out, st, oracle.render(s), hashes=True)
