"""The per-bin depth sort (stage 1 of the two-stage sort, Sec. 2, Stage 3, Phase 2), read
back from the workspace after a render: every bin's reference list must be strictly
ascending (the keys are distinct: representative depth, then quad index), hold each
(quad, bin) pair at most once, and only name visible quads whose pixel box meets the bin.
The image does not show a wrong order (the exact path repairs every misordered pixel), so
these lists are checked directly, on scenes that take every branch of the sort: a few
references, register-sorted runs of 64, 128 and 256 keys with zero to five merge levels, the
dense-bin bucket sort, the merge in shared memory alone (equal depths) and the merge through
global memory.
"""
import numpy as np
import pytest
import torch

import scenegen
from tests.scene_helpers import rects_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import paper_2405_13364_gb300 as P
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    P.load_library()
    return P


def _bin_lists(lr, s, k=3):
    from paper_2405_13364_gb300 import _binding as B
    r = lr.Renderer(sorter_k=k)
    ds = lr.DeviceScene.from_scene(s)
    out = r.make_outputs(s.width, s.height)
    view = r.view_struct(ds, s.width, s.height, out)
    r.render_views([view])
    torch.cuda.synchronize()
    st = r.stats()
    lay = B.lr_workspace_layout(r.ctx, [view], r._ws_bytes)
    ws = r._ws
    off = ((int(ws.data_ptr()) + 255) & ~255) - int(ws.data_ptr())

    def grab(o, nbytes, dtype):
        return ws[off + o: off + o + nbytes].cpu().numpy().view(dtype)

    nb = int(lay.total_bins)
    bin_off = grab(lay.bin_off, 4 * (nb + 1), np.uint32).astype(np.int64)
    total = int(bin_off[-1])
    refs = grab(lay.refs, 8 * total, np.uint64)
    q = s.num_quads
    rect = grab(lay.rec_rect, 8 * q, np.uint32).reshape(q, 2)
    r.close()
    return st, bin_off, refs, rect


def _check(s, st, bin_off, refs, rect, bin_px=32):
    assert st["status"] == 0
    nbx = (s.width + bin_px - 1) // bin_px
    nb = len(bin_off) - 1
    assert int(bin_off[-1]) == st["bin_refs"]
    lens = np.diff(bin_off)
    assert lens.max() == st["max_bin_refs"]
    for b in range(nb):
        lst = refs[bin_off[b]:bin_off[b + 1]]
        if len(lst) == 0:
            continue
        assert np.all(lst[1:] > lst[:-1]), f"bin {b}: list of {len(lst)} not strictly ascending"
        quads = (~(lst & np.uint64(0xFFFFFFFF))).astype(np.uint32).astype(np.int64)
        assert len(np.unique(quads)) == len(quads)
        assert quads.max() < s.num_quads
        rx, ry = rect[quads, 0], rect[quads, 1]
        px0, px1 = rx & 0xFFFF, rx >> 16
        py0, py1 = ry & 0xFFFF, ry >> 16
        bx, by = b % nbx, b // nbx
        assert np.all(px0 != 0xFFFF)   # visible quads only
        assert np.all((px0 <= bx * bin_px + bin_px - 1) & (px1 >= bx * bin_px))
        assert np.all((py0 <= by * bin_px + bin_px - 1) & (py1 >= by * bin_px))
    return lens


def _particles_in_one_bin(n, seed):
    return scenegen.gaussian_particles(n, 32, 32, seed=seed, sigma=1.5, size_px=(2.0, 4.0))


@pytest.mark.parametrize("n,branch", [(40, None), (200, None), (700, None), (1300, None), (1900, None),
                                      (6000, 0), (30000, 2)])
def test_one_bin_sorted(lr, n, branch):
    s = _particles_in_one_bin(n, seed=40 + n % 17)
    st, bin_off, refs, rect = _bin_lists(lr, s)
    lens = _check(s, st, bin_off, refs, rect)
    assert lens.sum() == st["quads_visible"]   # every square lies in the 32 x 32 image
    if branch is not None:
        assert st["sort_bins"][branch] == 1


def test_equal_depths_sorted(lr):
    # 2048..8192 references at one depth: the bucket sort gives up, the merge sort in shared
    # memory orders them by quad index alone
    rng = np.random.default_rng(23)
    rects = []
    for _ in range(4000):
        x0, y0 = rng.uniform(0, 24, 2)
        rects.append((float(np.floor(x0 * 4) / 4), float(np.floor(y0 * 4) / 4),
                      float(np.floor(x0 * 4) / 4 + 6.0), float(np.floor(y0 * 4) / 4 + 5.0)))
    cols = np.concatenate([rng.random((4000, 3)), rng.uniform(0.02, 0.2, (4000, 1))], 1)
    s = rects_scene(rects, width=32, height=32, colors=cols)
    st, bin_off, refs, rect = _bin_lists(lr, s)
    _check(s, st, bin_off, refs, rect)
    assert st["sort_bins"][1] == 1


def test_many_bins_sorted(lr):
    # a frame of many bins with lists of a few hundred references (two to five runs of 256)
    s = scenegen.wavy_layers(640, 360, 32, 96, 48, seed=3, color_mode=scenegen.COLOR_VERTEX)
    st, bin_off, refs, rect = _bin_lists(lr, s)
    lens = _check(s, st, bin_off, refs, rect)
    assert lens.max() > 256 and (lens > 0).sum() > 100
