"""Benchmark of the exact-OIT rasteriser on the 1920x1080 stacked-layer workload.

One step = one full frame through the whole pipeline (setup, binning, per-bin sort,
rasterisation with the per-pixel sorter, exact overflow path) of the 1080p workload:
32 wavy layers x 256x128 quads = 1,048,576 indexed quads, per-vertex RGBA, mean depth
complexity 24 (about 49.9M fragments per frame). Inputs are resident in HBM; the L2 is
flushed (a 512 MiB write) before every timed step and the flush is outside the timed
events. Prints one JSON line, which also carries the 1920x1080 particle frame (2M
flat-colour squares, depth complexity above 1,000) as the `particles` sub-object.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (the plain definition: gather, sort, composite
every pixel) on this host's cores on the same workload; under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms/frame & Gfrag/s at 1080p; served frames/s with p50/p99 latency"
WORKLOAD = "layers-1080p: 1920x1080, 32 wavy layers x 256x128 = 1,048,576 indexed quads, " \
           "per-vertex RGBA, mean depth complexity 24"
# algorithmic lane operations per fragment of the rasteriser: 3 edge tests (2 integer
# multiply-adds + 1 compare each) = 9, depth key = 2 int->fp32 conversions + 4 fp32
# multiplies + 2 adds = 8, sorter = K compare/selects, blend = 8 fp32 ops
OPS_PER_FRAG_BASE = 25
# kernels launched per frame (one view): k_init (which also writes the view descriptor),
# k_setup, k_bin_count, k_bin_scan, k_bin_scatter, k_bin_sort, k_bin_sort_big, k_raster,
# k_overflow
LAUNCHES_PER_FRAME = 9
# DRAM bytes (read + write) per k_raster launch from ncu captures (profiles/), keyed by
# (workload, K, carried colours), with the hash of the rasteriser sources they were taken
# on: the figure is reported only while the kernel is unchanged.
RASTER_TRAFFIC = {
    # (DRAM read + write bytes per launch, ncu smsp__issue_active, ncu smsp__inst_executed,
    #  source hash of the captured build)
    ("layers", 1, False): (101_893_120, 0.7544, 348_696_989, "3e9f8ff852bad3aa"),      # profiles/k_raster_layers1080p.md
    ("particles", 1, False): (383_102_464, 0.6758, 847_920_159, "3e9f8ff852bad3aa"),  # profiles/k_raster_particles1080p.md
}
# the same for the rasteriser's variants and the multisample resolve on the layer frame
# (K = 1): (DRAM bytes per launch, issue-slot share, warp instructions, kernel us, hash)
VARIANT_CAPTURES = {
    "alpha_threshold": (93_937_920, 0.7421, 273_373_076, 300.6, "3e9f8ff852bad3aa"),   # profiles/k_raster_alpha_layers1080p.md
    "lit": (116_687_360, 0.5619, 422_811_933, 605.7, "3e9f8ff852bad3aa"),               # profiles/k_raster_lit_layers1080p.md
    "msaa_resolve": (149_222_923, 0.2601, 7_452_000, 26.6, "3e9f8ff852bad3aa"),         # profiles/k_resolve_msaa4_layers1080p.md
}
RASTER_SOURCES = ("lr_raster.cuh", "lr_common.cuh")
LANES_PER_SM_CLK = 128
# the autotuner's candidates for the timed workloads: sorter capacity, bin size, rasteriser
# CTAs per SM (0 = the occupancy limit)
TUNE_KS = (1, 2, 3)
TUNE_BINS = (16, 32, 64)
TUNE_CTAS = (0, 2)
TUNE_BLOCKS = (4, 8)
TUNE_SHARED = (False, True)


def tune_label(t):
    """k<K>[c]_b<bin>[_cta<n>] for one autotuner candidate."""
    return (f"k{t['sorter_k']}{'c' if t['carry_colors'] else ''}_b{t['bin_size']}"
            + (f"_blk8x{t['block_h']}" if t.get("block_h", 4) != 4 else "")
            + ("_strip" if t.get("shared_setup") else "")
            + (f"_cta{t['raster_ctas_per_sm']}" if t["raster_ctas_per_sm"] else ""))


def _workloads():
    import scenegen
    return {
        "layers": ("layers-1080p: 1920x1080, 32 wavy layers x 256x128 = 1,048,576 indexed quads, "
                   "per-vertex RGBA, mean depth complexity 24", lambda s: scenegen.config_layers_1080p(seed=s)),
        "particles": ("particles-1080p: 1920x1080, 2,000,000 camera-facing quads 2-16 px, flat RGBA, "
                      "centre depth complexity > 500", lambda s: scenegen.config_particles_1080p(seed=s)),
        "frustum": ("frustum-256: 256x256, 2,000 random parallelograms, flat RGBA",
                    lambda s: scenegen.config_small_frustum(seed=s)),
        "diff": ("layers-1024: 1024x1024, 32 layers x 128x128 = 524,288 quads, flat RGBA",
                 lambda s: scenegen.config_diff_1024(seed=s)),
    }


class _LazyWorkloads(dict):
    def __missing__(self, key):
        self.update(_workloads())
        return dict.__getitem__(self, key)


WORKLOADS = _LazyWorkloads()


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")  # written by the environment, not by this repo
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return None


def raster_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2405_13364_gb300", "csrc")
    for f in RASTER_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def variant_capture(name: str):
    """The committed ncu figures of a rasteriser variant (or the resolve) as a dict, or None
    once the rasteriser's sources differ from the captured build."""
    t = VARIANT_CAPTURES.get(name)
    if t is None or t[4] != raster_source_hash():
        return None
    return {"dram_bytes_per_launch": t[0], "issue_active": t[1], "warp_instructions": t[2], "kernel_us": t[3],
            "source": "ncu capture, K = 1, layers-1080p frame (profiles/)"}


def raster_capture(workload: str, k: int, carry: bool, bin_size: int = 32, block_h: int = 4, shared: bool = False):
    """(traffic bytes, issue-slot utilisation, warp instructions) of the committed ncu
    capture of this rasteriser build (taken with 32-pixel bins), or Nones once the sources
    differ from it or the configuration is another."""
    t = RASTER_TRAFFIC.get((workload, k, carry))
    if t is None or t[3] != raster_source_hash() or bin_size != 32 or block_h != 4 or shared:
        return None, None, None
    return t[0], t[1], t[2]


class ClockSampler:
    """Samples SM clocks and throttle reasons during timing with one `nvidia-smi -lms`
    process (started before the timed region, stopped after it)."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 50):
        self.index = index
        self.period_ms = period_ms
        self.samples = []
        self._proc = None
        self._t = None

    def _read(self):
        for line in self._proc.stdout:
            f = [x.strip() for x in line.strip().split(",")]
            if len(f) >= 7:
                self.samples.append(f)

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.15)            # the first sample lands before the timed work starts
        except Exception:
            self._proc = None
        return self

    def __exit__(self, *a):
        if self._proc is not None:
            time.sleep(0.06)            # one more sample at the end of the timed region
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
            self._t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples), "period_ms": self.period_ms}


def frame_benchmark(P, torch, scene, k, carry, steps, warmup, flush, dev, dist=None, bin_size=32, ctas=0,
                    block_h=4, shared=False):
    """Device-timed frames of one workload: a renderer without per-stage events renders
    `steps` frames (L2 flushed before each, outside the events; CUDA events on the stream
    around each frame), then a second renderer that records an event between stages gives
    the per-stage breakdown from separate frames. Returns (ms per frame, first-frame stats,
    stage means, the outputs and view of the timed renderer)."""
    W, H = scene.width, scene.height
    ds = P.DeviceScene.from_scene(scene, device=dev)
    r = P.Renderer(sorter_k=k, carry_colors=carry, bin_size=bin_size, raster_ctas_per_sm=ctas, block_h=block_h,
                   shared_setup=shared)
    rt = P.Renderer(sorter_k=k, timing=True, carry_colors=carry, bin_size=bin_size, raster_ctas_per_sm=ctas,
                    block_h=block_h, shared_setup=shared)
    out = r.make_outputs(W, H)
    view = r.view_struct(ds, W, H, out)
    view_t = rt.view_struct(ds, W, H, out)
    # size the workspace once (retries on reference overflow), then render without checks
    r.render_views([view])
    st0 = r.stats()
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        r.render_views([view], check=False)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index or 0)
    with sampler:
        for i in range(steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            r.render_views([view], check=False)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    rt.render_views([view_t])
    stage_steps = min(steps, 20)
    stage_sum = {kk: 0.0 for kk in rt.stats()["stage_ms"]}
    for i in range(stage_steps):
        flush.fill_(i & 0xFF)
        rt.render_views([view_t], check=False)
        st = rt.stats()                 # synchronises; per-stage CUDA events of this frame
        for kk, v in st["stage_ms"].items():
            stage_sum[kk] += v
    rt.close()
    ms = [a.elapsed_time(b) for a, b in ev]
    stages = {kk: round(v / stage_steps, 4) for kk, v in stage_sum.items()}
    return sum(ms) / len(ms), st0, stages, sampler, (r, ds, out, view)


def raster_roofline(workload, k, carry, frags, raster_ms, sm_count, sm_max_mhz, bin_size=32, block_h=4, shared=False):
    """The rasteriser against the plain-ALU peak: algorithmic lane operations per fragment
    (25 + K) x fragments / its CUDA-event time, against SMs x 128 lanes x the SM clock,
    with the SM count of the device the run is on; plus the instruction-issue ceiling of
    the committed ncu capture of the same build, when there is one."""
    ops = (OPS_PER_FRAG_BASE + k) * frags
    peak = sm_count * LANES_PER_SM_CLK * sm_max_mhz * 1e6 / 1e12   # T lane-ops/s
    achieved = ops / (raster_ms * 1e-3) / 1e12
    traffic, issue_active, inst = raster_capture(workload, k, carry, bin_size, block_h, shared)
    issue_ceiling = None
    if inst:
        ceil_gfrag = sm_count * 4 * sm_max_mhz * 1e6 / (inst / frags) / 1e9
        got = frags / (raster_ms * 1e-3) / 1e9
        issue_ceiling = {"warp_instructions_per_fragment": round(inst / frags, 3),
                         "ceiling_gfrag_s": round(ceil_gfrag, 1), "achieved_gfrag_s": round(got, 1),
                         "frac": round(got / ceil_gfrag, 4)}
    return {"bound": "alu", "kernel": "k_raster", "achieved": round(achieved, 4), "peak": round(peak, 3),
            "unit": "Tlane-op/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "ncu_issue_active": issue_active, "ops_per_fragment": OPS_PER_FRAG_BASE + k,
            "raster_ms": raster_ms,
            "peak_basis": f"{sm_count} SMs x 128 lanes x {sm_max_mhz:.0f} MHz (max SM clock)",
            "issue_ceiling": issue_ceiling}


def particles_benchmark(P, torch, args, flush, dev, sm_count, hbm_gbs):
    """The 1920x1080 particle frame (2,000,000 flat-colour squares, centre depth complexity
    above 1,000) beside the headline: frame time, Gfrag/s, per-stage times, the rasteriser's
    roofline and the setup / binning HBM fractions, with the autotuned sorter capacity."""
    import scenegen
    from paper_2405_13364_gb300 import autotune
    scene = scenegen.config_particles_1080p()
    ds = P.DeviceScene.from_scene(scene, device=dev)
    tuned = autotune.tune(ds, scene.width, scene.height, ks=TUNE_KS, ctas_per_sm=TUNE_CTAS, reps=3, device=dev,
                          bin_sizes=TUNE_BINS, block_hs=TUNE_BLOCKS, shared=TUNE_SHARED, use_cache=False)
    del ds
    k, carry = tuned["sorter_k"], bool(tuned.get("carry_colors"))
    ms, st0, stages, sampler, (r, _, _, _) = frame_benchmark(P, torch, scene, k, carry, min(args.steps, 20),
                                                             args.warmup, flush, dev, None, tuned["bin_size"],
                                                             tuned["raster_ctas_per_sm"], tuned["block_h"],
                                                             bool(tuned["shared_setup"]))
    r.close()
    frags = st0["fragments"]
    clocks = sampler.summary()
    return {"workload": WORKLOADS["particles"][0], "frame": f"{scene.width}x{scene.height}",
            "quads": scene.num_quads, "fragments_per_frame": frags, "ms_per_frame": round(ms, 4),
            "gfrag_s": round(frags / (ms * 1e-3) / 1e9, 3), "sorter_k": k, "carry_colors": carry,
            "bin_size": tuned["bin_size"], "raster_ctas_per_sm": tuned["raster_ctas_per_sm"],
            "block": f"8x{tuned['block_h']}", "shared_setup": bool(tuned["shared_setup"]),
            "autotune_ms": {tune_label(t): round(t["ms"], 4) for t in tuned["table"]},
            "stage_ms": stages, "overflow_pixels": st0["overflow_pixels"], "bins_high": st0["bins_high"],
            "sort_bins": st0["sort_bins"],
            "roofline": raster_roofline("particles", k, carry, frags, stages["raster"], sm_count,
                                        clocks.get("sm_max_mhz") or 2070.0, tuned["bin_size"], tuned["block_h"],
                                        bool(tuned["shared_setup"])),
            **stage_rooflines(scene, st0, stages, hbm_gbs), "clocks": clocks}


def stage_rooflines(scene, st0, stages, hbm_gbs):
    """Setup and binning against the HBM copy bandwidth, two ways: by the algorithmic bytes
    of the method (indices 16 B per quad, positions 12 B per vertex, a 52-byte record per
    visible quad (snapped XY 32 B, 1/w 16 B, bin rectangle 4 B) and a 4-byte id per quad for
    setup; for binning 4 B per visible quad read by each of the two passes, 4 B per
    reference written, 8 B per bin), and by the bytes this implementation's kernels move
    (16 B indices + 12 B per vertex + 80 B of records per quad for setup; 12 B read by the
    count and 16 B by the scatter per quad, 8 B per reference, 16 B per bin for binning)."""
    W, H = scene.width, scene.height
    nq, nv = scene.num_quads, scene.num_vertices
    vis = int(st0["quads_visible"])
    refs = int(st0["bin_refs"])
    bins = ((W + 31) // 32) * ((H + 31) // 32)
    idx = 16 * nq if scene.indices is not None else 0
    setup_alg = idx + 12 * nv + 52 * vis + 4 * nq
    setup_impl = idx + 12 * nv + 80 * nq
    bin_alg = 2 * 4 * vis + 4 * refs + 8 * bins
    bin_impl = 28 * nq + 8 * refs + 16 * bins
    out = {}
    for name, ms, alg, impl in (("setup_hbm", stages.get("setup"), setup_alg, setup_impl),
                                ("binning_hbm", (stages.get("count") or 0) + (stages.get("scan") or 0)
                                 + (stages.get("scatter") or 0), bin_alg, bin_impl)):
        if not ms or not hbm_gbs:
            out[name] = None
            continue
        a = alg / (ms * 1e-3) / 1e9
        b = impl / (ms * 1e-3) / 1e9
        out[name] = {"ms": round(ms, 4), "algorithmic_bytes": alg, "achieved_gbs": round(a, 1),
                     "frac": round(a / hbm_gbs, 4), "implementation_bytes": impl,
                     "implementation_gbs": round(b, 1), "implementation_frac": round(b / hbm_gbs, 4),
                     "peak_gbs": hbm_gbs, "peak_basis": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    return out


def serving_benchmark(P, torch, num_requests=256, rate_hz=200.0, seed=0):
    """The served render stream: a seeded Poisson trace of mixed requests (resolutions
    256x256 .. 2560x1440, the three scene generators at quad counts log-uniform in
    10k-2M), served by the continuous-batching server, against the same trace served one
    lr_render at a time. Every request renders with the sorter capacity the autotuner
    picks for its size bucket (GPU, resolution, quad count and colour mode, each rounded
    to a power of two), in both forms. Scenes are built and uploaded before the clock
    starts: layer requests get their own grid scaled to the quad count; particle and
    frustum requests take the first N quads of one 2M-quad scene per generator and
    resolution, which has the same distribution as a fresh N-quad scene (quads are drawn
    independently). Returns a dict."""
    import time as _time

    import numpy as np

    import scenegen
    from paper_2405_13364_gb300 import autotune
    trace = scenegen.request_trace(num_requests, rate_hz, seed=seed)
    base = {}

    def scene_of(req):
        kind, q, w, h = req["kind"], req["quads"], req["width"], req["height"]
        if kind == "layers":
            return P.DeviceScene.from_scene(scenegen.scene_for_request(req))
        key = (kind, w, h)
        if key not in base:
            big = dict(req, quads=2_000_000, seed=7)
            base[key] = P.DeviceScene.from_scene(scenegen.scene_for_request(big))
        b = base[key]
        return P.DeviceScene(b.positions[: 4 * q], None, b.colors[:q], b.color_mode, b.view_proj, b.near, b.far)

    scenes = [scene_of(r) for r in trace]
    # the autotuned sorter capacity of every request's size bucket (tuned once per bucket,
    # on the bucket's first request)
    ks, tuned_buckets = [], {}
    for sc, q in zip(scenes, trace):
        key = autotune.workload_key(q["width"], q["height"], sc.num_quads, sc.color_mode)
        if key not in tuned_buckets:
            tuned_buckets[key] = autotune.tune(sc, q["width"], q["height"], ks=(1, 2, 3), reps=3,
                                               carry=(False,), use_cache=False)["sorter_k"]
        ks.append(tuned_buckets[key])
    frags = 0
    # ---- sequential: one lr_render per request, in arrival order, one at a time -----------
    r = P.Renderer(sorter_k=3)
    outs = [r.make_outputs(q["width"], q["height"]) for q in trace]
    views = [P.Renderer.view_struct(s, q["width"], q["height"], o, sorter_k=k)
             for s, q, o, k in zip(scenes, trace, outs, ks)]
    for v in views[:8]:
        r.render_views([v])                      # warm-up, sizes the workspace
    ref_imgs = []
    seq_lat, t_start = [], None
    t0 = _time.perf_counter()
    for q, v, o in zip(trace, views, outs):
        now = _time.perf_counter() - t0
        if now < q["arrival"]:
            _time.sleep(q["arrival"] - now)
        st = r.render_views([v])                 # synchronises and checks the status
        done = _time.perf_counter() - t0
        seq_lat.append(done - q["arrival"])
        frags += int(st.fragments)
    seq_span = (_time.perf_counter() - t0)
    ref_imgs = [o["rgba"].clone() for o in outs]
    # saturated: everything queued at once
    t1 = _time.perf_counter()
    for v in views:
        r.render_views([v])
    seq_sat = _time.perf_counter() - t1
    r.close()
    # ---- served: continuous batching ---------------------------------------------------------
    srv = P.Server(sorter_k=3, num_slots=3, max_batch_views=8, slot_workspace_bytes=2 << 30)
    warm = [srv.submit(scenes[i], trace[i]["width"], trace[i]["height"], sorter_k=ks[i]) for i in range(8)]
    for t in warm:
        while srv.poll(t, timeout_us=100_000) is None:
            pass

    def serve(arrivals):
        souts = [srv.renderer.make_outputs(q["width"], q["height"]) for q in trace]
        tickets, t_sub = [], []
        base = P.Server.now_ns()
        tb = _time.perf_counter()
        for i, q in enumerate(trace):
            if arrivals:
                now = _time.perf_counter() - tb
                if now < q["arrival"]:
                    _time.sleep(q["arrival"] - now)
            tickets.append(srv.submit(scenes[i], q["width"], q["height"], out=souts[i], sorter_k=ks[i]))
        lat, last_done = [], 0
        for i, t in enumerate(tickets):
            res = None
            while res is None:
                res = srv.poll(t, timeout_us=200_000)
            status, _, info = res
            assert status == 0, status
            arr_ns = base + int((trace[i]["arrival"] if arrivals else 0.0) * 1e9)
            lat.append((info["done_ns"] - arr_ns) * 1e-9)
            last_done = max(last_done, info["done_ns"])
        return souts, lat, (last_done - base) * 1e-9

    souts, srv_lat, srv_span = serve(True)
    torch.cuda.synchronize()
    same = all(torch.equal(a["rgba"], b) for a, b in zip(souts, ref_imgs))
    _, _, srv_sat = serve(False)
    st = srv.stats()
    srv.close()
    pct = lambda xs, p: float(np.percentile(np.array(xs) * 1e3, p))
    return {
        "trace": f"{num_requests} requests, Poisson {rate_hz:.0f} req/s, seed {seed}",
        "fragments": frags,
        "served": {"fps": round(num_requests / srv_span, 1), "p50_ms": round(pct(srv_lat, 50), 3),
                   "p99_ms": round(pct(srv_lat, 99), 3),
                   "saturated_fps": round(num_requests / srv_sat, 1),
                   "batches": st["batches"], "mean_views_per_batch": round(st["batched_views"] / max(1, st["batches"]), 2)},
        "sequential": {"fps": round(num_requests / seq_span, 1), "p50_ms": round(pct(seq_lat, 50), 3),
                       "p99_ms": round(pct(seq_lat, 99), 3), "saturated_fps": round(num_requests / seq_sat, 1)},
        "served_equals_sequential_bitwise": bool(same),
        "sorter_k_per_request": {f"k{k}": ks.count(k) for k in sorted(set(ks))},
        "size_buckets_tuned": len(tuned_buckets),
        "quads_per_request": {"min": min(s_.num_quads for s_ in scenes), "max": max(s_.num_quads for s_ in scenes),
                              "total": sum(s_.num_quads for s_ in scenes)},
    }


def differentiable_benchmark(P, torch, steps: int, sorter_k: int = 1):
    """Differentiable compositing on the 1024x1024 layer scene (524,288 quads, flat RGBA):
    each step renders the image, forms dL/dC = 2 (C - T) for the squared L2 distance to a
    target rendered with perturbed colours, and runs the backward (per-quad RGBA
    gradients, bins and per-pixel order recomputed; the forward's exact-path mask spares the
    backward its detection pass), all on the device. Reports forward, backward and step
    times (CUDA events)."""
    import scenegen
    s = scenegen.config_diff_1024()
    ds = P.DeviceScene.from_scene(s)
    r = P.Renderer(sorter_k=sorter_k)
    tgt = r.render(ds.with_colors(torch.tensor(scenegen.perturbed_target_colors(s.colors, seed=1),
                                               device=ds.colors.device)), s.width, s.height)["rgba"]
    # the forward also writes its exact-path mask, which spares the backward its detection pass
    out = r.make_outputs(s.width, s.height, exact_mask=True)
    view = r.view_struct(ds, s.width, s.height, out)
    st = r.render_views([view])                        # sizes the workspace
    frags = int(st.fragments)
    g = torch.zeros_like(out["rgba"])
    r.render_backward(ds, s.width, s.height, out["rgba"], g, exact_mask=out["exact_mask"])
    stream = torch.cuda.current_stream()
    fwd, bwd = [], []
    for i in range(steps + 3):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        r.render_views([view], check=False)
        g[..., :3] = 2.0 * (out["rgba"][..., :3] - tgt[..., :3])
        e1.record(stream)
        r.render_backward(ds, s.width, s.height, out["rgba"], g, check=False, exact_mask=out["exact_mask"])
        e2.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            fwd.append(e0.elapsed_time(e1))
            bwd.append(e1.elapsed_time(e2))
    st = P._binding.lr_get_stats(r.ctx, raise_on_error=False)
    if st.status != 0:
        raise RuntimeError(f"differentiable benchmark: backward status {st.status}")
    r.close()
    f, b = statistics.median(fwd), statistics.median(bwd)
    return {"workload": "1024x1024, 524,288 quads (layer generator, flat RGBA), loss = squared L2 to a "
                        "target with RGBA + N(0, 0.05)",
            "fragments": frags, "forward_ms": round(f, 4), "backward_ms": round(b, 4),
            "step_ms": round(f + b, 4), "backward_gfrag_s": round(frags / (b * 1e-3) / 1e9, 2),
            "steps": steps, "sorter_k": sorter_k}


def run_reference(args):
    """The CPU oracle on this host's cores, same workload and metric."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    import oracle
    import scenegen
    scene = scenegen.config_layers_1080p()
    cores = oracle.num_threads(0)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.render(scene)
    times, frags = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.render(scene)
        times.append(time.perf_counter() - t0)
        frags = r["stats"]["fragments"]
    ms = 1e3 * sum(times) / len(times)
    value = frags / (ms * 1e-3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Gfrag/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frame": "1920x1080", "quads": scene.num_quads,
                   "fragments_per_frame": frags},
        "cpu_baseline": {"value": round(value, 4), "unit": "Gfrag/s", "cores": cores, "kind": "oracle",
                         "sample": f"full 1920x1080 frame x {args.steps} steps"},
        "e2e": {"value": round(value, 4), "unit": "Gfrag/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2405_13364_gb300 as P
    import scenegen
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)

    scene = WORKLOADS[args.workload][1](rank)
    W, H = scene.width, scene.height
    ds = P.DeviceScene.from_scene(scene, device=dev)
    tuned = None
    if args.k == 0:
        # the sorter capacity K picked by the autotuner for this workload (any K gives the
        # same exact result; it only moves pixels between the sorter and the exact path)
        from paper_2405_13364_gb300 import autotune
        tuned = autotune.tune(ds, W, H, ks=TUNE_KS, ctas_per_sm=TUNE_CTAS, reps=3, device=dev,
                              bin_sizes=TUNE_BINS, block_hs=TUNE_BLOCKS, shared=TUNE_SHARED, use_cache=False)
        args.k = tuned["sorter_k"]
    carry = bool(tuned and tuned.get("carry_colors"))
    bin_size = tuned["bin_size"] if tuned else 32
    ctas = tuned["raster_ctas_per_sm"] if tuned else 0
    block_h = tuned["block_h"] if tuned else 4
    shared = bool(tuned["shared_setup"]) if tuned else False
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ms_frame, st0, stages, sampler, (r, ds, out, view) = frame_benchmark(
        P, torch, scene, args.k, carry, args.steps, args.warmup, flush, dev, dist, bin_size, ctas, block_h, shared)
    frags = st0["fragments"]
    from paper_2405_13364_gb300 import replicas
    ms_step = replicas.max_over_ranks(ms_frame, dist, dev)
    if dist:
        dist.barrier()
    value = world * frags / (ms_step * 1e-3) / 1e9

    # ---- end to end through the public API with host buffers -----------------------------
    # HostStream: every step copies the scene in from pinned host memory and the image
    # back out; the copies of neighbouring frames overlap rendering (two streams of copies,
    # two device buffers each way). The serial variant (copy in, render, copy out, wait)
    # is reported beside it.
    host_pos = torch.from_numpy(scene.positions).pin_memory()
    host_idx = None if scene.indices is None else torch.from_numpy(scene.indices.view(np.int32)).pin_memory()
    host_col = torch.from_numpy(scene.colors).pin_memory()
    host_out = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
    h2d = host_pos.numel() * 4 + (0 if host_idx is None else host_idx.numel() * 4) + host_col.numel() * 4
    d2h = host_out.numel() * 4
    hs = P.HostStream(r, host_pos.shape[0], scene.num_quads, host_idx is not None, scene.color_mode,
                      host_col.shape[0], W, H)
    vp = ds.view_proj
    for _ in range(3):
        hs.submit(host_pos, host_idx, host_col, vp, ds.near, ds.far, host_out)
    hs.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(hs.s_in)
    hs.s_render.wait_event(t_start)
    hs.s_out.wait_event(t_start)
    for i in range(args.steps):
        hs.submit(host_pos, host_idx, host_col, vp, ds.near, ds.far, host_out)
    hs.s_in.wait_stream(hs.s_out)
    t_end.record(hs.s_in)
    hs.synchronize()
    e2e_ms = replicas.max_over_ranks(t_start.elapsed_time(t_end) / args.steps, dist, dev)
    e2e_value = world * frags / (e2e_ms * 1e-3) / 1e9

    dpos, dcol = hs.pos[0], hs.col[0]
    didx = hs.idx[0]
    e_scene = P.DeviceScene(dpos, didx, dcol, scene.color_mode, ds.view_proj, ds.near, ds.far)
    e_out = r.make_outputs(W, H)
    e_view = r.view_struct(e_scene, W, H, e_out)

    def e2e_serial_step():
        dpos.copy_(host_pos, non_blocking=True)
        if didx is not None:
            didx.copy_(host_idx, non_blocking=True)
        dcol.copy_(host_col, non_blocking=True)
        r.render_views([e_view], check=False)
        host_out.copy_(e_out["rgba"], non_blocking=True)

    torch.cuda.synchronize()
    for _ in range(2):
        e2e_serial_step()
    torch.cuda.synchronize()
    e_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_serial_step()
        b.record(stream)
        torch.cuda.synchronize()
        e_ms.append(a.elapsed_time(b))
    e2e_serial_ms = replicas.max_over_ranks(sum(e_ms) / len(e_ms), dist, dev)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    serving = None
    differentiable = None
    if args.workload == "layers" and world == 1 and not args.no_serving:
        serving = serving_benchmark(P, torch)
        differentiable = differentiable_benchmark(P, torch, steps=20)

    clocks = sampler.summary()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline = raster_roofline(args.workload, args.k, carry, frags, stages["raster"], sm_count,
                               clocks.get("sm_max_mhz") or 2070.0, bin_size, block_h, shared)
    peaks = _measured_peaks()
    hbm = peaks.get("hbm_gbs") if peaks else None
    particles = None
    if args.workload == "layers" and world == 1 and not args.no_particles:
        particles = particles_benchmark(P, torch, args, flush, dev, sm_count, hbm)

    # pixels that needed the exact path, per sorter capacity (the paper's Sec. 3 error rates
    # are for pixels left misordered; here they are recomputed exactly)
    overflow_frac = {}
    if world == 1:
        for kk in (1, 3, 8, 12):
            rk = P.Renderer(sorter_k=kk)
            ok_ = rk.make_outputs(W, H)
            stk = rk.render_views([rk.view_struct(ds, W, H, ok_)])
            overflow_frac[f"k{kk}"] = round(int(stk.overflow_pixels) / (W * H), 6)
            rk.close()

    # ---- the opt-in alpha threshold (lossy, Sec. 3 "Alpha threshold"): frame time beside
    # the exact frame's, and the largest deviation from the exact image (at most 1/128) ---
    alpha_threshold = None
    if world == 1:
        ra = P.Renderer(sorter_k=args.k, carry_colors=carry, alpha_threshold=True, bin_size=bin_size,
                        raster_ctas_per_sm=ctas)
        oa = ra.make_outputs(W, H)
        va = ra.view_struct(ds, W, H, oa)
        ra.render_views([va])
        sta = ra.stats()
        for _ in range(args.warmup):
            ra.render_views([va], check=False)
        a_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(20)]
        torch.cuda.synchronize()
        for i, (a0, a1) in enumerate(a_ev):
            flush.fill_(i & 0xFF)
            a0.record(stream)
            ra.render_views([va], check=False)
            a1.record(stream)
        torch.cuda.synchronize()
        a_ms = sum(a0.elapsed_time(a1) for a0, a1 in a_ev) / len(a_ev)
        dev_max = float((oa["rgba"] - out["rgba"]).abs().max().item())
        alpha_threshold = {"t_min": 1 / 128, "ms_per_frame": round(a_ms, 4),
                           "speedup_vs_exact": round(ms_step / a_ms, 3),
                           "fragments_evaluated": int(sta["fragments"]), "fragments_exact": frags,
                           "overflow_pixels": int(sta["overflow_pixels"]),
                           "max_abs_deviation_from_exact": round(dev_max, 6), "bound": 1 / 128,
                           "ncu": variant_capture("alpha_threshold")}
        ra.close()

    # ---- multisampling (4 samples per pixel, every sample an exact composite) ------------
    msaa = None
    if world == 1:
        rm = P.Renderer(sorter_k=args.k, carry_colors=carry, bin_size=bin_size, raster_ctas_per_sm=ctas)
        rm.render_msaa(ds, W, H, samples=4)           # sizes the workspace
        stm = rm.stats()
        for _ in range(args.warmup):
            rm.render_msaa(ds, W, H, samples=4, check=False)
        m_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(10)]
        torch.cuda.synchronize()
        for i, (a0, a1) in enumerate(m_ev):
            flush.fill_(i & 0xFF)
            a0.record(stream)
            rm.render_msaa(ds, W, H, samples=4, check=False)
            a1.record(stream)
        torch.cuda.synchronize()
        m_ms = sum(a0.elapsed_time(a1) for a0, a1 in m_ev) / len(m_ev)
        msaa = {"samples": 4, "ms_per_frame": round(m_ms, 4),
                "sample_fragments_per_frame": int(stm["fragments"]),
                "gfrag_s": round(int(stm["fragments"]) / (m_ms * 1e-3) / 1e9, 2),
                "vs_single_sample_ms": round(m_ms / ms_step, 3), "ncu_resolve": variant_capture("msaa_resolve")}
        rm.close()

    # ---- lit colours (per-vertex normals, one directional light) on the same layers ------
    lit = None
    if world == 1 and args.workload == "layers":
        lscene = scenegen.wavy_layers(color_mode=scenegen.COLOR_LIT)
        lds = P.DeviceScene.from_scene(lscene, device=dev)
        rl = P.Renderer(sorter_k=args.k, carry_colors=carry, bin_size=bin_size, raster_ctas_per_sm=ctas)
        rl.set_lighting(lscene.light[:3], lscene.light[3])
        ol = rl.make_outputs(W, H)
        vl = rl.view_struct(lds, W, H, ol)
        rl.render_views([vl])
        for _ in range(args.warmup):
            rl.render_views([vl], check=False)
        l_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(20)]
        torch.cuda.synchronize()
        for i, (a0, a1) in enumerate(l_ev):
            flush.fill_(i & 0xFF)
            a0.record(stream)
            rl.render_views([vl], check=False)
            a1.record(stream)
        torch.cuda.synchronize()
        l_ms = sum(a0.elapsed_time(a1) for a0, a1 in l_ev) / len(l_ev)
        lit = {"ms_per_frame": round(l_ms, 4), "gfrag_s": round(frags / (l_ms * 1e-3) / 1e9, 2),
               "vs_unlit_ms": round(l_ms / ms_step, 3),
               "shading": "per fragment: perspective-correct normal, two-sided Lambert + ambient",
               "ncu": variant_capture("lit")}
        rl.close()
        del lds

    # ---- CPU oracle on a bounded sample: full frames for ~10 s ---------------------------
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        cores = oracle.num_threads(0)
        t0 = time.perf_counter()
        n_frames, cfrags = 0, 0
        while time.perf_counter() - t0 < 8.0 or n_frames == 0:
            cfrags += oracle.render(scene)["stats"]["fragments"]
            n_frames += 1
        dt = time.perf_counter() - t0
        cpu = {"value": round(cfrags / dt / 1e9, 4), "unit": "Gfrag/s", "cores": cores, "kind": "oracle",
               "sample": f"{n_frames} full 1920x1080 frames ({dt:.1f} s)"}
        small = scenegen.config_small_frustum()
        t1 = []
        for _ in range(3):
            a = time.perf_counter()
            oracle.render(small, nthreads=1)
            t1.append(time.perf_counter() - a)
        cpu["small_frustum_single_thread_ms"] = round(1e3 * statistics.median(t1), 2)

    line = {
        "metric": METRIC if args.workload == "layers" else f"Gfrag/s ({args.workload})",
        "value": round(value, 3), "unit": "Gfrag/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][0], "frame": f"{W}x{H}", "quads": scene.num_quads,
                   "fragments_per_frame": frags, "sorter_k": args.k,
                   "carry_colors": carry,
                   "bin_size": bin_size, "raster_ctas_per_sm": ctas, "block": f"8x{block_h}", "shared_setup": shared,
                   "autotune_ms": None if tuned is None else {tune_label(t): round(t["ms"], 4) for t in tuned["table"]},
                   "l2": "flushed before every step (512 MiB write, outside the timed events)",
                   "parallelism": f"replicas x{world} (one frame per GPU per step)"},
        "stage_ms": stages,
        "overflow_pixels": st0["overflow_pixels"],
        "roofline": roofline,
        **stage_rooflines(scene, st0, stages, hbm),
        "particles": particles,
        "overflow_pixel_fraction": overflow_frac,
        "alpha_threshold": alpha_threshold,
        "msaa": msaa,
        "lit": lit,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 3), "unit": "Gfrag/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 4),
                "api": "HostStream (copies of neighbouring frames overlap rendering)",
                "serial_ms_per_step": round(e2e_serial_ms, 4)},
        "served_stream": serving,
        "differentiable": differentiable,
        "gpu_launches": LAUNCHES_PER_FRAME * args.steps,
        "clocks": clocks,
    }
    if peaks:
        line["measured_peaks"] = {"hbm_gbs": peaks.get("hbm_gbs")}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_profile(args):
    """A short, self-contained run for ncu: a few frames of one workload, no timing, no CPU
    baseline. --variant picks the rasteriser form: exact (the benchmark's), alpha (the
    opt-in alpha threshold), lit (lit per-vertex colours on the layer scene) or msaa (4
    samples per pixel, ending in k_resolve). Kernel launch order per exact frame: k_init,
    k_setup, k_bin_count, k_bin_scan, k_bin_scatter, k_bin_sort, k_bin_sort_big, k_raster,
    k_overflow."""
    import torch

    import paper_2405_13364_gb300 as P
    import scenegen
    torch.cuda.set_device(0)
    if args.variant == "lit":
        scene = scenegen.wavy_layers(color_mode=scenegen.COLOR_LIT)
    else:
        scene = {"layers": scenegen.config_layers_1080p, "particles": scenegen.config_particles_1080p,
                 "frustum": scenegen.config_small_frustum, "diff": scenegen.config_diff_1024}[args.workload]()
    r = P.Renderer(sorter_k=args.k, alpha_threshold=args.variant == "alpha")
    if args.variant == "lit":
        r.set_lighting(scene.light[:3], scene.light[3])
    ds = P.DeviceScene.from_scene(scene)
    if args.variant == "msaa":
        r.render_msaa(ds, scene.width, scene.height, samples=4)
        for _ in range(args.steps):
            r.render_msaa(ds, scene.width, scene.height, samples=4, check=False)
    else:
        out = r.make_outputs(scene.width, scene.height)
        view = r.view_struct(ds, scene.width, scene.height, out)
        r.render_views([view])
        for _ in range(args.steps):
            r.render_views([view], check=False)
    torch.cuda.synchronize()
    st = r.stats()
    print(json.dumps({"profile_workload": args.workload, "variant": args.variant, "frames": args.steps + 1,
                      "fragments": st["fragments"], "overflow_pixels": st["overflow_pixels"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--k", type=int, default=0, help="sorter capacity K; 0 = autotuned")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-particles", action="store_true", help="skip the particle-frame sub-object")
    ap.add_argument("--profile", action="store_true", help="short run for ncu (see run_profile)")
    ap.add_argument("--variant", default="exact", choices=["exact", "alpha", "lit", "msaa"],
                    help="rasteriser form of the --profile run")
    ap.add_argument("--workload", default="layers", choices=["layers", "particles", "frustum", "diff"])
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
