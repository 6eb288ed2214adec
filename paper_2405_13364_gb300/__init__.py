"""GB300-native exact order-independent-transparency quad rasteriser (LucidRaster,
arXiv 2405.13364): Python layer over the C ABI in include/lr.h.

PyTorch is used for device memory and streams only; every pipeline stage runs in the
CUDA library (liblr.so). Nothing here computes pixels.

    r = Renderer(sorter_k=3)
    scene = DeviceScene.from_arrays(positions, indices, colors, color_mode, view_proj, near, far)
    out = r.render(scene, 1920, 1080)          # {'rgba': f32[H][W][4] on the GPU, ...}
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import _binding as B
from ._binding import (LR_COLOR_FLAT, LR_COLOR_LIT, LR_COLOR_VERTEX, LR_ERR_OVERFLOW, LR_FLAG_TIMING, LR_OK,
                       LrError, lr_camera, lr_config, lr_quads, lr_stats, lr_target, lr_view)

__all__ = ["Renderer", "DeviceScene", "HostStream", "Server", "LrError", "LR_COLOR_FLAT", "LR_COLOR_VERTEX",
           "LR_COLOR_LIT",
           "composite", "load_library"]


def load_library():
    """Load (and if needed build) liblr.so; raises if the CUDA library is unavailable."""
    return B.load()


def _ptr(t):
    return 0 if t is None else int(t.data_ptr())


@dataclasses.dataclass
class DeviceScene:
    """A quad scene resident on the GPU (tensors are kept alive by this object)."""

    positions: torch.Tensor            # f32[V][3]
    indices: torch.Tensor | None       # i32/u32[Q][4] or None
    colors: torch.Tensor               # f32[Q][4], f32[V][4], or f32[V][8] (lit: RGBA, normal, unused)
    color_mode: int
    view_proj: tuple                   # 16 floats, row-major
    near: float
    far: float

    @property
    def num_quads(self) -> int:
        return int(self.indices.shape[0]) if self.indices is not None else int(self.positions.shape[0] // 4)

    @classmethod
    def from_arrays(cls, positions, indices, colors, color_mode, view_proj, near, far,
                    device="cuda"):
        def dev(a, dtype):
            t = torch.as_tensor(a)
            if t.dtype != dtype:
                t = t.to(dtype)
            return t.to(device).contiguous()

        pos = dev(positions, torch.float32).reshape(-1, 3)
        idx = None
        if indices is not None:
            idx_t = torch.as_tensor(indices)
            if idx_t.dtype != torch.int32:
                idx_t = idx_t.to(torch.int64).to(torch.int32)
            idx = idx_t.to(device).contiguous().reshape(-1, 4)
        col = dev(colors, torch.float32).reshape(-1, 8 if int(color_mode) == B.LR_COLOR_LIT else 4)
        vp = tuple(float(x) for x in torch.as_tensor(view_proj, dtype=torch.float32).reshape(-1).tolist())
        return cls(pos, idx, col, int(color_mode), vp, float(near), float(far))

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        """From any object with positions / indices / colors / color_mode / view_proj /
        near / far attributes (e.g. the seeded generators' Scene)."""
        return cls.from_arrays(scene.positions, scene.indices, scene.colors, scene.color_mode,
                               scene.view_proj, scene.near, scene.far, device=device)

    def with_colors(self, colors: torch.Tensor) -> "DeviceScene":
        return dataclasses.replace(self, colors=colors.contiguous())

    def quads_struct(self) -> lr_quads:
        return lr_quads(_ptr(self.positions), int(self.positions.shape[0]), _ptr(self.indices),
                        self.num_quads, _ptr(self.colors), self.color_mode, 0)

    def camera_struct(self) -> lr_camera:
        cam = lr_camera()
        for i, v in enumerate(self.view_proj):
            cam.view_proj[i] = v
        cam.near_z = self.near
        cam.far_z = self.far
        return cam


class Outputs(dict):
    """Per-view outputs: 'rgba' and optionally 'rgba8', 'count', 'hash' (device tensors)."""


class Renderer:
    """Owns an lr_ctx and a growable workspace on one CUDA device."""

    def __init__(self, sorter_k: int = 3, max_width: int = 2560, max_height: int = 2048,
                 timing: bool = False, ref_factor: int = 4, raster_ctas_per_sm: int = 0,
                 device=None, carry_colors: bool = False, alpha_threshold: bool = False,
                 bin_size: int = 32, block_h: int = 4, shared_setup: bool = False):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        B.load()
        with torch.cuda.device(self.device):
            flags = ((LR_FLAG_TIMING if timing else 0) | (B.LR_FLAG_CARRY_COLORS if carry_colors else 0)
                     | (B.LR_FLAG_ALPHA_THRESHOLD if alpha_threshold else 0))
            cfg = lr_config(max_width, max_height, sorter_k, raster_ctas_per_sm, ref_factor,
                            flags, self.device.index, bin_size, block_h, int(shared_setup))
            self.ctx = B.lr_create(cfg)
        self.sorter_k = sorter_k
        self.bin_size = bin_size
        self.block_h = block_h
        self.shared_setup = shared_setup
        self._ws = None
        self._ws_bytes = 0

    def set_lighting(self, light_dir, ambient: float):
        """Light of lit scenes (LR_COLOR_LIT) rendered from now on: direction toward the
        light in world space (any length) and the ambient term in [0, 1]."""
        B.lr_set_lighting(self.ctx, light_dir, ambient)

    def close(self):
        if getattr(self, "ctx", None):
            B.lr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- workspace -----------------------------------------------------------------------
    def workspace(self, nbytes: int):
        """A 256-byte aligned device buffer of at least nbytes (grown, never shrunk)."""
        if self._ws is None or self._ws_bytes < nbytes:
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            self._ws_bytes = nbytes
        base = int(self._ws.data_ptr())
        return (base + 255) & ~255, self._ws_bytes

    # ---- views -----------------------------------------------------------------------------
    def make_outputs(self, width, height, rgba8=False, count=False, hash=False, exact_mask=False) -> Outputs:
        o = Outputs()
        o["rgba"] = torch.empty((height, width, 4), dtype=torch.float32, device=self.device)
        if exact_mask:   # one 32-bit word per 8x4 half-block
            o["exact_mask"] = torch.empty(((height + 3) // 4, (width + 7) // 8), dtype=torch.int32,
                                          device=self.device)
        if rgba8:
            o["rgba8"] = torch.empty((height, width, 4), dtype=torch.uint8, device=self.device)
        if count:
            o["count"] = torch.empty((height, width), dtype=torch.int32, device=self.device)
        if hash:
            o["hash"] = torch.empty((height, width), dtype=torch.int64, device=self.device)
        return o

    @staticmethod
    def view_struct(scene: DeviceScene, width: int, height: int, out: Outputs,
                    owned_tiles: torch.Tensor | None = None, sorter_k: int = 0) -> lr_view:
        """owned_tiles: None, or a device int32/uint32 tensor holding the bit set of the
        32x32-pixel tiles to rasterise (partition.owned_bitset's layout); the other tiles'
        pixels of every output are left as they are. sorter_k: 0 for the renderer's sorter
        capacity, else this view's (all views of one batch must agree)."""
        tgt = lr_target(_ptr(out["rgba"]), _ptr(out.get("rgba8")), _ptr(out.get("count")),
                        _ptr(out.get("hash")), _ptr(out.get("exact_mask")))
        if owned_tiles is not None:
            ntiles = ((width + 31) // 32) * ((height + 31) // 32)
            if owned_tiles.numel() < (ntiles + 31) // 32 or owned_tiles.element_size() != 4 \
                    or not owned_tiles.is_cuda or not owned_tiles.is_contiguous():
                raise ValueError("owned_tiles: a contiguous device tensor of ceil(tiles / 32) 32-bit words")
        return lr_view(scene.quads_struct(), scene.camera_struct(), width, height, tgt, _ptr(owned_tiles),
                       int(sorter_k), 0)

    def render_views(self, views, stream=None, check: bool = True):
        """Render lr_view structs with one lr_render_batch call; grows the workspace and
        retries once if binning needed more references than the workspace held."""
        stream = torch.cuda.current_stream(self.device) if stream is None else stream
        need = B.lr_workspace_size_batch(self.ctx, views)
        for _ in range(3):
            ptr, nbytes = self.workspace(need)
            B.lr_render_batch(self.ctx, views, ptr, nbytes, stream.cuda_stream)
            if not check:
                return None
            st = B.lr_get_stats(self.ctx, raise_on_error=False)
            if st.status == LR_ERR_OVERFLOW:
                need = B.lr_workspace_size_refs(self.ctx, views, int(st.bin_refs * 1.25) + 1024)
                continue
            if st.status != LR_OK:
                raise LrError(st.status, B.lr_last_error(self.ctx))
            return st
        raise LrError(LR_ERR_OVERFLOW, "bin references kept exceeding the workspace")

    def render(self, scene: DeviceScene, width: int, height: int, rgba8=False, count=False,
               hash=False, stream=None, check: bool = True, exact_mask=False, owned_tiles=None,
               out: Outputs | None = None) -> Outputs:
        """owned_tiles: see view_struct. out: outputs to render into (default: new ones)."""
        if out is None:
            out = self.make_outputs(width, height, rgba8, count, hash, exact_mask)
        self.render_views([self.view_struct(scene, width, height, out, owned_tiles)], stream, check)
        return out

    def render_msaa(self, scene: DeviceScene, width: int, height: int, samples: int = 4, offsets=None,
                    stream=None, check: bool = True) -> torch.Tensor:
        """Multisampled render (lr_render_msaa): every sample position of a pixel gets its own
        exact composite and the pixel is their mean. offsets: None for the default pattern of
        4 or 16 samples, else samples pairs (dx, dy) from the pixel centre in 1/256 px."""
        stream = torch.cuda.current_stream(self.device) if stream is None else stream
        out = torch.empty((height, width, 4), dtype=torch.float32, device=self.device)
        need = B.lr_workspace_size_msaa(self.ctx, scene.num_quads, width, height, samples)
        for _ in range(3):
            ptr, nbytes = self.workspace(need)
            B.lr_render_msaa(self.ctx, scene.quads_struct(), scene.camera_struct(), width, height, samples,
                             offsets, _ptr(out), ptr, nbytes, stream.cuda_stream)
            if not check:
                return out
            st = B.lr_get_stats(self.ctx, raise_on_error=False)
            if st.status == LR_ERR_OVERFLOW:      # more bin references than the workspace held
                need = nbytes + 20 * int(st.bin_refs) + (1 << 20)
                continue
            if st.status != LR_OK:
                raise LrError(st.status, B.lr_last_error(self.ctx))
            return out
        raise LrError(LR_ERR_OVERFLOW, "bin references kept exceeding the workspace")

    def render_batch(self, items, stream=None, check: bool = True, **outputs):
        """items: list of (DeviceScene, width, height). One launch per stage for all."""
        outs = [self.make_outputs(w, h, **outputs) for _, w, h in items]
        views = [self.view_struct(s, w, h, o) for (s, w, h), o in zip(items, outs)]
        self.render_views(views, stream, check)
        return outs

    def capture(self, items, stream=None, **outputs) -> "GraphBatch":
        """Capture a multi-view render of items [(DeviceScene, width, height)] into a CUDA
        graph on a workspace of its own; replays may swap scenes/cameras of equal shape."""
        return GraphBatch(self, items, stream, **outputs)

    def stats(self) -> dict:
        st = B.lr_get_stats(self.ctx, raise_on_error=False)
        names = ["setup", "count", "scan", "scatter", "sort", "raster", "overflow", "total"]
        return dict(status=st.status, n_views=st.n_views, quads_in=st.quads_in,
                    quads_visible=st.quads_visible, culled=list(st.culled), bin_refs=st.bin_refs,
                    bin_refs_capacity=st.bin_refs_capacity, bins_nonempty=st.bins_nonempty,
                    bins_high=st.bins_high, max_bin_refs=st.max_bin_refs, fragments=st.fragments,
                    overflow_pixels=st.overflow_pixels, sort_bins=list(st.sort_bins),
                    stage_ms={n: st.stage_ms[i] for i, n in enumerate(names)})

    # ---- differentiation ----------------------------------------------------------------------
    def render_backward(self, scene: DeviceScene, width: int, height: int, fwd_rgba: torch.Tensor,
                        grad_out: torch.Tensor, stream=None, check: bool = True,
                        exact_mask: torch.Tensor | None = None) -> torch.Tensor:
        """dL/d(flat per-quad RGBA) given dL/d(image); the fragment order is recomputed.
        exact_mask: the forward's `exact_mask` output (render(..., exact_mask=True)) for the
        same scene and renderer, which saves the detection pass; if it does not match, the
        call is repeated without it (with check=True)."""
        stream = torch.cuda.current_stream(self.device) if stream is None else stream
        grad = torch.zeros((scene.num_quads, 4), dtype=torch.float32, device=self.device)
        fwd_rgba = fwd_rgba.contiguous()
        grad_out = grad_out.to(torch.float32).contiguous()
        out = Outputs(rgba=fwd_rgba)
        view = self.view_struct(scene, width, height, out)
        need = B.lr_workspace_size_batch(self.ctx, [view])
        for _ in range(3):
            ptr, nbytes = self.workspace(need)
            B.lr_render_backward(self.ctx, scene.quads_struct(), scene.camera_struct(), width, height,
                                 _ptr(fwd_rgba), _ptr(grad_out), _ptr(exact_mask), _ptr(grad), ptr, nbytes,
                                 stream.cuda_stream)
            if not check:
                return grad
            st = B.lr_get_stats(self.ctx, raise_on_error=False)
            if st.status == B.LR_ERR_MASK_MISMATCH:
                exact_mask = None
                grad.zero_()
                continue
            if st.status == LR_ERR_OVERFLOW:
                need = B.lr_workspace_size_refs(self.ctx, [view], int(st.bin_refs * 1.25) + 1024)
                grad.zero_()
                continue
            if st.status != LR_OK:
                raise LrError(st.status, B.lr_last_error(self.ctx))
            return grad
        raise LrError(LR_ERR_OVERFLOW, "bin references kept exceeding the workspace")


class GraphBatch:
    """A captured multi-view render (lr_graph_create / lr_graph_launch)."""

    def __init__(self, renderer: Renderer, items, stream=None, **outputs):
        self.r = renderer
        self.items = list(items)
        self.outs = [renderer.make_outputs(w, h, **outputs) for _, w, h in self.items]
        self.views = [Renderer.view_struct(s, w, h, o) for (s, w, h), o in zip(self.items, self.outs)]
        # size the workspace with one checked render (grows it on reference overflow)
        renderer.render_views(self.views, stream)
        need = renderer._ws_bytes
        self._ws = torch.empty(need + 256, dtype=torch.uint8, device=renderer.device)
        self._ptr = (int(self._ws.data_ptr()) + 255) & ~255
        torch.cuda.synchronize(renderer.device)
        self.graph = B.lr_graph_create(renderer.ctx, self.views, self._ptr, need)

    def launch(self, items=None, stream=None):
        """Replay; items (same shapes as captured) replaces scenes/cameras/outputs."""
        stream = torch.cuda.current_stream(self.r.device) if stream is None else stream
        views = None
        if items is not None:
            self.items = list(items)
            views = [Renderer.view_struct(s, w, h, o) for (s, w, h), o in zip(self.items, self.outs)]
            self.views = views
        B.lr_graph_launch(self.r.ctx, self.graph, views, stream.cuda_stream)
        return self.outs

    def close(self):
        if self.graph:
            torch.cuda.synchronize(self.r.device)
            B.lr_graph_destroy(self.graph)
            self.graph = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostStream:
    """Renders scenes that live in host memory, frame after frame, overlapping each
    frame's host->device copy of its inputs and the previous frame's device->host read of
    its image with rendering. Inputs and outputs are host tensors (pinned for overlap);
    every frame is copied in and its image copied out. One copy stream each way, the
    renderer on its own stream, `depth` device buffers each way.

        hs = HostStream(renderer, num_vertices, num_quads, indexed, color_mode, num_colors,
                        width, height)
        hs.submit(pos, idx, col, view_proj, near, far, out)   # returns at once
        hs.synchronize()                                       # out holds the image
    """

    def __init__(self, renderer: "Renderer", num_vertices: int, num_quads: int, indexed: bool,
                 color_mode: int, num_colors: int, width: int, height: int, depth: int = 2):
        self.r = renderer
        self.dev = renderer.device
        self.width, self.height = int(width), int(height)
        self.color_mode = int(color_mode)
        self.depth = int(depth)
        self.pos = [torch.empty((num_vertices, 3), dtype=torch.float32, device=self.dev) for _ in range(depth)]
        self.idx = [torch.empty((num_quads, 4), dtype=torch.int32, device=self.dev) if indexed else None
                    for _ in range(depth)]
        cw = 8 if color_mode == B.LR_COLOR_LIT else 4
        self.col = [torch.empty((num_colors, cw), dtype=torch.float32, device=self.dev) for _ in range(depth)]
        self.out = [renderer.make_outputs(width, height) for _ in range(depth)]
        self.s_in = torch.cuda.Stream(self.dev)
        self.s_render = torch.cuda.Stream(self.dev)
        self.s_out = torch.cuda.Stream(self.dev)
        ev = lambda: [torch.cuda.Event() for _ in range(depth)]
        self.in_done, self.render_done, self.out_done = ev(), ev(), ev()
        self.started = [False] * depth
        self.sized = False
        self.i = 0

    def submit(self, pos, idx, col, view_proj, near, far, out: torch.Tensor):
        """Queue one frame: pos f32[V][3], idx i32[Q][4] or None, col f32[Q or V][4] and
        out f32[H][W][4] are host tensors (pinned for asynchronous copies)."""
        k = self.i % self.depth
        self.i += 1
        if self.started[k]:
            self.s_in.wait_event(self.render_done[k])     # the slot's inputs are free again
        with torch.cuda.stream(self.s_in):
            self.pos[k].copy_(pos, non_blocking=True)
            if self.idx[k] is not None:
                self.idx[k].copy_(idx, non_blocking=True)
            self.col[k].copy_(col, non_blocking=True)
            self.in_done[k].record(self.s_in)
        self.s_render.wait_event(self.in_done[k])
        if self.started[k]:
            self.s_render.wait_event(self.out_done[k])    # the slot's image was read back
        vp = view_proj if isinstance(view_proj, tuple) and len(view_proj) == 16 else \
            tuple(float(x) for x in torch.as_tensor(view_proj, dtype=torch.float32).reshape(-1).tolist())
        scene = DeviceScene(self.pos[k], self.idx[k], self.col[k], self.color_mode, vp, float(near), float(far))
        view = Renderer.view_struct(scene, self.width, self.height, self.out[k])
        # the first frame sizes the workspace (a checked render, which waits for it); later
        # frames of the same shape reuse it, and synchronize() reports a failed one
        self.r.render_views([view], stream=self.s_render, check=not self.sized)
        self.sized = True
        self.render_done[k].record(self.s_render)
        self.s_out.wait_event(self.render_done[k])
        with torch.cuda.stream(self.s_out):
            out.copy_(self.out[k]["rgba"], non_blocking=True)
            self.out_done[k].record(self.s_out)
        self.started[k] = True

    def synchronize(self):
        """Wait for every queued frame; raises LrError if the last render failed (e.g. a
        frame that needed more bin references than the first frame sized)."""
        self.s_in.synchronize()
        self.s_render.synchronize()
        self.s_out.synchronize()
        st = B.lr_get_stats(self.r.ctx, raise_on_error=False)
        if st.status != LR_OK:
            raise LrError(st.status, B.lr_last_error(self.r.ctx))


class _Composite(torch.autograd.Function):
    @staticmethod
    def forward(actx, colors, renderer, scene, width, height):
        s = scene.with_colors(colors.detach().to(torch.float32).contiguous())
        res = renderer.render(s, width, height, exact_mask=True)
        out = res["rgba"]
        actx.renderer, actx.scene, actx.size = renderer, s, (width, height)
        actx.save_for_backward(out, res["exact_mask"])
        return out

    @staticmethod
    def backward(actx, grad_out):
        out, mask = actx.saved_tensors
        w, h = actx.size
        g = actx.renderer.render_backward(actx.scene, w, h, out, grad_out, exact_mask=mask)
        return g, None, None, None, None


def composite(colors: torch.Tensor, renderer: Renderer, scene: DeviceScene, width: int,
              height: int) -> torch.Tensor:
    """Differentiable render w.r.t. flat per-quad RGBA colors f32[Q][4] (CUDA tensor).
    Coverage and depth order are exact and piecewise constant: they get no gradient."""
    return _Composite.apply(colors, renderer, scene, width, height)


class Server:
    """Continuous-batching render server (lr_server_start / lr_submit / lr_poll).

    Owns its own context (created with the renderer options given here). Submitted
    scenes and outputs are kept alive until their request completes.
    """

    def __init__(self, sorter_k: int = 3, num_slots: int = 2, max_batch_views: int = 16,
                 slot_workspace_bytes: int = 512 << 20, poll_interval_us: int = 20,
                 max_width: int = 2560, max_height: int = 2048, device=None, light=None,
                 idle_spin_us: int = 0):
        self.renderer = Renderer(sorter_k=sorter_k, max_width=max_width, max_height=max_height,
                                 device=device)
        self.ctx = self.renderer.ctx
        if light is not None:      # (x, y, z) toward the light, ambient: for lit requests
            self.renderer.set_lighting(light[:3], light[3])
        cfg = B.lr_server_config(num_slots, max_batch_views, slot_workspace_bytes, poll_interval_us, idle_spin_us)
        B.lr_server_start(self.ctx, cfg)
        self._live = {}
        self.running = True

    def submit(self, scene: DeviceScene, width: int, height: int, out: Outputs | None = None,
               sorter_k: int = 0, **outputs) -> int:
        """sorter_k: 0 for the server's capacity, else this request's (e.g. autotuned for its
        size); the server batches requests of equal capacity only."""
        out = out if out is not None else self.renderer.make_outputs(width, height, **outputs)
        view = Renderer.view_struct(scene, width, height, out, sorter_k=sorter_k)
        t = B.lr_submit(self.ctx, view)
        self._live[t] = (scene, out)
        return t

    def poll(self, ticket: int, timeout_us: int = 0):
        """None while pending; else (status, outputs, info dict with ns timestamps)."""
        st, res, info = B.lr_poll_info(self.ctx, ticket, timeout_us)
        if st != LR_OK:
            return None
        _, out = self._live.pop(ticket)
        return res, out, dict(submit_ns=info.submit_ns, launch_ns=info.launch_ns,
                              done_ns=info.done_ns, batch_views=info.batch_views)

    def stats(self) -> dict:
        st = B.lr_server_get_stats(self.ctx)
        return {n: getattr(st, n) for n, _ in B.lr_server_stats._fields_}

    @staticmethod
    def now_ns() -> int:
        return B.lr_now_ns()

    def stop(self):
        if self.running:
            B.lr_server_stop(self.ctx)
            self.running = False

    def close(self):
        self.stop()
        self.renderer.close()
