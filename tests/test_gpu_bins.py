"""Every bin size (16, 32, 64 pixels; lr_config.bin_size) against the oracle: the image,
per-pixel fragment counts and coverage hashes do not depend on it (counts and hashes
bit-exact, colour within 1e-5), including dense bins that take each branch of the
high-density sort, ragged frame sizes, owned-tile sets and the 1920x1080 workloads."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from paper_2405_13364_gb300 import partition as PT

pytestmark = pytest.mark.gpu

COLOR_TOL = 1e-5


@pytest.fixture(scope="module")
def lr():
    import paper_2405_13364_gb300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    P.load_library()
    return P


def _render(lr, s, bin_size, k=3, owned=None, out=None):
    r = lr.Renderer(sorter_k=k, bin_size=bin_size)
    if out is None:
        out = r.make_outputs(s.width, s.height, rgba8=True, count=True, hash=True)
    r.render(lr.DeviceScene.from_scene(s), s.width, s.height, owned_tiles=owned, out=out)
    torch.cuda.synchronize()
    st = r.stats()
    r.close()
    return out, st


def _compare(out, st, o, mask=None):
    sel = (slice(None),) if mask is None else (mask,)
    cnt = out["count"].cpu().numpy().view(np.uint32)
    hsh = out["hash"].cpu().numpy().view(np.uint64)
    rgba = out["rgba"].cpu().numpy()
    np.testing.assert_array_equal(cnt[sel], o["count"][sel])
    np.testing.assert_array_equal(hsh[sel], o["hash"][sel])
    d = np.abs(rgba[sel].astype(np.float64) - o["rgba"][sel]).max()
    assert d <= COLOR_TOL, d
    if mask is None:
        d8 = np.abs(out["rgba8"].cpu().numpy().astype(np.int32) - o["rgba8"].astype(np.int32)).max()
        assert d8 <= 1
        assert st["fragments"] == int(o["count"].sum())


def _scenes():
    return {
        "frustum_ragged": scenegen.frustum_parallelograms(3000, 200, 141, seed=4),
        "layers_vertex": scenegen.wavy_layers(333, 190, layers=32, nx=48, ny=24, seed=1),
        "particles": scenegen.gaussian_particles(60_000, 320, 180, seed=3),
        "big_near_quads": scenegen.frustum_parallelograms(300, 160, 96, seed=9, edge_range=(0.5, 6.0), far=8.0),
        "tiny": scenegen.frustum_parallelograms(40, 13, 7, seed=2, edge_range=(0.5, 3.0), far=10.0),
    }


@pytest.mark.parametrize("bin_size", [16, 64])
@pytest.mark.parametrize("name", list(_scenes()))
@pytest.mark.parametrize("k", [1, 3])
def test_bin_size_matches_oracle(lr, bin_size, name, k):
    s = _scenes()[name]
    out, st = _render(lr, s, bin_size, k)
    assert st["status"] == 0
    _compare(out, st, oracle.render(s))


@pytest.mark.parametrize("bin_size", [16, 64])
def test_dense_bins_every_sort_branch(lr, bin_size):
    # one bin holding > 20480 references with distinct depths (global merge), a bin of
    # 2048..20480 (bucket sort), and equal depths (the bucket sort gives up)
    s = scenegen.gaussian_particles(40_000, bin_size, bin_size, seed=31, sigma=1.5, size_px=(2.0, 4.0))
    out, st = _render(lr, s, bin_size)
    assert st["bins_high"] >= 1 and st["sort_bins"][2] >= 1
    _compare(out, st, oracle.render(s))
    s = scenegen.gaussian_particles(8_000, 2 * bin_size, bin_size, seed=32, sigma=2.0, size_px=(2.0, 4.0))
    out, st = _render(lr, s, bin_size)
    assert st["sort_bins"][0] >= 1
    _compare(out, st, oracle.render(s))


@pytest.mark.parametrize("bin_size", [16, 64])
def test_bin_size_with_owned_tiles(lr, bin_size):
    s = scenegen.wavy_layers(333, 190, layers=16, nx=40, ny=20, seed=6)
    o = oracle.render(s)
    owner = PT.assign_tiles(s.width, s.height, 3)
    for rank in range(3):
        bits = torch.from_numpy(PT.owned_bitset(owner, rank).view(np.int32)).cuda()
        r = lr.Renderer(sorter_k=3, bin_size=bin_size)
        out = r.make_outputs(s.width, s.height, rgba8=True, count=True, hash=True)
        out["rgba"].fill_(float("nan"))
        r.render(lr.DeviceScene.from_scene(s), s.width, s.height, owned_tiles=bits, out=out)
        torch.cuda.synchronize()
        r.close()
        mine = np.zeros((s.height, s.width), bool)
        for x0, y0, x1, y1 in PT.tile_rects(owner, rank, s.width, s.height):
            mine[y0:y1, x0:x1] = True
        _compare(out, None, o, mine)
        assert np.isnan(out["rgba"].cpu().numpy()[~mine]).all()


@pytest.mark.parametrize("bin_size", [16, 64])
@pytest.mark.parametrize("name", ["layers", "particles"])
def test_bin_size_full_size(lr, bin_size, name):
    s = {"layers": scenegen.config_layers_1080p, "particles": scenegen.config_particles_1080p}[name]()
    out, st = _render(lr, s, bin_size, k=1)
    assert st["status"] == 0
    _compare(out, st, oracle.render(s))


def test_bin_size_refused():
    import paper_2405_13364_gb300 as P
    with pytest.raises(P.LrError):
        P.Renderer(bin_size=24)
