"""The autotuner times sorter capacities, bin sizes and CTA counts, requires every candidate's image
to agree within 1e-5 (the pipeline is exact for any K), and caches its choice."""
import pytest

import scenegen

pytestmark = pytest.mark.gpu


def test_autotune_small(tmp_path, monkeypatch):
    import paper_2405_13364_gb300 as P
    from paper_2405_13364_gb300 import autotune
    monkeypatch.setenv("LR_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    s = scenegen.wavy_layers(320, 180, layers=16, nx=24, ny=12, seed=3)
    ds = P.DeviceScene.from_scene(s)
    res = autotune.tune(ds, s.width, s.height, ks=(1, 2, 3, 8), ctas_per_sm=(0, 1), reps=2,
                        bin_sizes=(16, 32, 64), block_hs=(4, 8), shared=(False, True))
    assert res["sorter_k"] in (1, 2, 3, 8) and res["bin_size"] in (16, 32, 64)
    # per-vertex colours (no colour-carrying variant): 4 K x 2 CTA counts x 3 bin sizes for
    # 8x4 half-blocks, 3 K (8x8 is built up to K = 3) x 2 x 3 for 8x8 blocks, 3 K x 2 for
    # the strip form (32-pixel bins only)
    assert len(res["table"]) == 24 + 18 + 6
    assert {t["bin_size"] for t in res["table"]} == {16, 32, 64}
    assert {t["block_h"] for t in res["table"]} == {4, 8} and any(t["shared_setup"] for t in res["table"])
    # K = 1 cannot order interpenetrating layers by itself: more exact-path pixels
    by_k = {t["sorter_k"]: t["overflow_pixels"] for t in res["table"]
            if t["raster_ctas_per_sm"] == 0 and t["bin_size"] == 32 and t["block_h"] == 4 and not t["shared_setup"]}
    assert by_k[1] >= by_k[8]
    again = autotune.tune(ds, s.width, s.height, ks=(1,), reps=1)
    assert again["sorter_k"] == res["sorter_k"]          # served from the cache
