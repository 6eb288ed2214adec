"""ctypes binding of the C ABI declared in include/lr.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards plain
pointers and sizes. The library must be built (``paper_2405_13364_gb300._build``); there
is no fallback: loading fails loudly if liblr.so is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

LR_OK = 0
LR_PENDING = 1
LR_ERR_INVALID_ARG = -1
LR_ERR_TOO_LARGE = -2
LR_ERR_OOM = -3
LR_ERR_CUDA = -4
LR_ERR_TIMEOUT = -5
LR_ERR_OVERFLOW = -6
LR_ERR_UNSUPPORTED = -7
LR_ERR_MASK_MISMATCH = -8

STATUS_NAMES = {0: "LR_OK", 1: "LR_PENDING", -1: "LR_ERR_INVALID_ARG", -2: "LR_ERR_TOO_LARGE",
                -3: "LR_ERR_OOM", -4: "LR_ERR_CUDA", -5: "LR_ERR_TIMEOUT", -6: "LR_ERR_OVERFLOW",
                -7: "LR_ERR_UNSUPPORTED", -8: "LR_ERR_MASK_MISMATCH"}

LR_COLOR_FLAT = 0
LR_COLOR_VERTEX = 1
LR_COLOR_LIT = 2
LR_FLAG_TIMING = 1
LR_FLAG_CARRY_COLORS = 2
LR_FLAG_NO_PDL = 4
LR_FLAG_ALPHA_THRESHOLD = 8


class LrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lr_config(ctypes.Structure):
    _fields_ = [("max_width", ctypes.c_int32), ("max_height", ctypes.c_int32),
                ("sorter_k", ctypes.c_int32), ("raster_ctas_per_sm", ctypes.c_int32),
                ("ref_factor", ctypes.c_int32), ("flags", ctypes.c_int32), ("device", ctypes.c_int32),
                ("bin_size", ctypes.c_int32), ("block_h", ctypes.c_int32), ("shared_setup", ctypes.c_int32)]


class lr_quads(ctypes.Structure):
    _fields_ = [("positions", ctypes.c_void_p), ("num_vertices", ctypes.c_int64),
                ("indices", ctypes.c_void_p), ("num_quads", ctypes.c_int64),
                ("colors", ctypes.c_void_p), ("color_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class lr_camera(ctypes.Structure):
    _fields_ = [("view_proj", ctypes.c_float * 16), ("near_z", ctypes.c_float),
                ("far_z", ctypes.c_float)]


class lr_target(ctypes.Structure):
    _fields_ = [("rgba", ctypes.c_void_p), ("rgba8", ctypes.c_void_p),
                ("frag_count", ctypes.c_void_p), ("cov_hash", ctypes.c_void_p),
                ("exact_mask", ctypes.c_void_p)]


class lr_view(ctypes.Structure):
    _fields_ = [("quads", lr_quads), ("camera", lr_camera), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("target", lr_target), ("owned_tiles", ctypes.c_void_p),
                ("sorter_k", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class lr_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_views", ctypes.c_int32),
                ("quads_in", ctypes.c_int64), ("quads_visible", ctypes.c_int64),
                ("culled", ctypes.c_int64 * 8), ("bin_refs", ctypes.c_int64),
                ("bin_refs_capacity", ctypes.c_int64), ("bins_nonempty", ctypes.c_int64),
                ("bins_high", ctypes.c_int64), ("max_bin_refs", ctypes.c_int64),
                ("fragments", ctypes.c_int64), ("overflow_pixels", ctypes.c_int64),
                ("stage_ms", ctypes.c_float * 8), ("sort_bins", ctypes.c_int64 * 3)]


class lr_ws_layout(ctypes.Structure):
    _fields_ = [("rec", ctypes.c_size_t), ("rec_rect", ctypes.c_size_t),
                ("rec_info", ctypes.c_size_t), ("bin_count", ctypes.c_size_t),
                ("bin_off", ctypes.c_size_t), ("refs", ctypes.c_size_t),
                ("total_quads", ctypes.c_int64), ("total_bins", ctypes.c_int64),
                ("refs_capacity", ctypes.c_int64)]


class lr_server_config(ctypes.Structure):
    _fields_ = [("num_slots", ctypes.c_int32), ("max_batch_views", ctypes.c_int32),
                ("slot_workspace_bytes", ctypes.c_int64), ("poll_interval_us", ctypes.c_int32),
                ("idle_spin_us", ctypes.c_int32)]


class lr_request_info(ctypes.Structure):
    _fields_ = [("submit_ns", ctypes.c_uint64), ("launch_ns", ctypes.c_uint64),
                ("done_ns", ctypes.c_uint64), ("batch_views", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class lr_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "batches",
                                             "batched_views", "split_batches", "queued")]


# every entry point declared in include/lr.h, with its ctypes signature
_P = ctypes.c_void_p
_SIGNATURES = {
    "lr_create": (ctypes.c_int, [ctypes.POINTER(lr_config), ctypes.POINTER(_P)]),
    "lr_destroy": (ctypes.c_int, [_P]),
    "lr_set_lighting": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_float]),
    "lr_workspace_size": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_size_t)]),
    "lr_workspace_size_batch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(lr_view),
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "lr_workspace_size_refs": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(lr_view),
                                              ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "lr_render": (ctypes.c_int, [_P, ctypes.POINTER(lr_quads), ctypes.POINTER(lr_camera),
                                 ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_size_t, _P]),
    "lr_render_batch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(lr_view), _P,
                                       ctypes.c_size_t, _P]),
    "lr_render_backward": (ctypes.c_int, [_P, ctypes.POINTER(lr_quads), ctypes.POINTER(lr_camera),
                                          ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P,
                                          ctypes.c_size_t, _P]),
    "lr_workspace_layout": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(lr_view),
                                           ctypes.c_size_t, ctypes.POINTER(lr_ws_layout)]),
    "lr_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(lr_stats)]),
    "lr_last_error": (ctypes.c_char_p, [_P]),
    "lr_server_start": (ctypes.c_int, [_P, ctypes.POINTER(lr_server_config)]),
    "lr_server_stop": (ctypes.c_int, [_P]),
    "lr_submit": (ctypes.c_int, [_P, ctypes.POINTER(lr_view), ctypes.POINTER(ctypes.c_uint64)]),
    "lr_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int)]),
    "lr_poll_info": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(lr_request_info)]),
    "lr_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(lr_server_stats)]),
    "lr_now_ns": (ctypes.c_uint64, []),
    "lr_graph_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(lr_view), _P, ctypes.c_size_t,
                                       ctypes.POINTER(_P)]),
    "lr_graph_launch": (ctypes.c_int, [_P, ctypes.POINTER(lr_view), _P]),
    "lr_graph_destroy": (ctypes.c_int, [_P]),
    "lr_render_noalloc": (ctypes.c_int, [ctypes.POINTER(lr_quads), ctypes.POINTER(lr_camera),
                                         ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "lr_workspace_size_msaa": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "lr_render_msaa": (ctypes.c_int, [_P, ctypes.POINTER(lr_quads), ctypes.POINTER(lr_camera),
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P,
                                      ctypes.c_size_t, _P]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblr.so (building it first when missing and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(ctx, status: int, what: str):
    if status != LR_OK:
        msg = load().lr_last_error(ctx) if ctx else b""
        raise LrError(status, f"{what}: {(msg or b'').decode(errors='replace')}")


def lr_create(config: lr_config | None = None):
    lib = load()
    out = _P()
    st = lib.lr_create(ctypes.byref(config) if config is not None else None, ctypes.byref(out))
    _check(None, st, "lr_create")
    return out


def lr_destroy(ctx):
    _check(None, load().lr_destroy(ctx), "lr_destroy")


def lr_workspace_size(ctx, num_quads: int, width: int, height: int) -> int:
    n = ctypes.c_size_t()
    _check(ctx, load().lr_workspace_size(ctx, num_quads, width, height, ctypes.byref(n)),
           "lr_workspace_size")
    return n.value


def lr_workspace_size_batch(ctx, views) -> int:
    arr = (lr_view * len(views))(*views)
    n = ctypes.c_size_t()
    _check(ctx, load().lr_workspace_size_batch(ctx, len(views), arr, ctypes.byref(n)),
           "lr_workspace_size_batch")
    return n.value


def lr_workspace_size_refs(ctx, views, bin_refs: int) -> int:
    arr = (lr_view * len(views))(*views)
    n = ctypes.c_size_t()
    _check(ctx, load().lr_workspace_size_refs(ctx, len(views), arr, bin_refs, ctypes.byref(n)),
           "lr_workspace_size_refs")
    return n.value


def lr_render(ctx, quads: lr_quads, camera: lr_camera, width: int, height: int, out_rgba: int,
              workspace: int, workspace_bytes: int, stream: int):
    _check(ctx, load().lr_render(ctx, ctypes.byref(quads), ctypes.byref(camera), width, height,
                                 out_rgba, workspace, workspace_bytes, stream), "lr_render")


def lr_render_batch(ctx, views, workspace: int, workspace_bytes: int, stream: int):
    arr = (lr_view * len(views))(*views)
    _check(ctx, load().lr_render_batch(ctx, len(views), arr, workspace, workspace_bytes, stream),
           "lr_render_batch")


def lr_set_lighting(ctx, light_dir, ambient: float):
    d = (ctypes.c_float * 3)(*[float(v) for v in light_dir])
    _check(ctx, load().lr_set_lighting(ctx, d, float(ambient)), "lr_set_lighting")


def lr_workspace_size_msaa(ctx, num_quads: int, width: int, height: int, n_samples: int) -> int:
    n = ctypes.c_size_t(0)
    _check(ctx, load().lr_workspace_size_msaa(ctx, num_quads, width, height, n_samples, ctypes.byref(n)),
           "lr_workspace_size_msaa")
    return n.value


def lr_render_msaa(ctx, quads: lr_quads, camera: lr_camera, width: int, height: int, n_samples: int,
                   offsets, out_rgba: int, workspace: int, workspace_bytes: int, stream: int):
    """offsets: None (the default pattern) or a sequence of (dx, dy) in 1/256 px."""
    arr = None
    if offsets is not None:
        flat = [int(v) for xy in offsets for v in xy]
        arr = (ctypes.c_int32 * len(flat))(*flat)
    _check(ctx, load().lr_render_msaa(ctx, ctypes.byref(quads), ctypes.byref(camera), width, height, n_samples,
                                      arr, out_rgba, workspace, workspace_bytes, stream), "lr_render_msaa")


def lr_render_backward(ctx, quads: lr_quads, camera: lr_camera, width: int, height: int,
                       fwd_rgba: int, grad_out: int, exact_mask: int, grad_colors: int, workspace: int,
                       workspace_bytes: int, stream: int):
    _check(ctx, load().lr_render_backward(ctx, ctypes.byref(quads), ctypes.byref(camera), width,
                                          height, fwd_rgba, grad_out, exact_mask, grad_colors,
                                          workspace, workspace_bytes, stream), "lr_render_backward")


def lr_workspace_layout(ctx, views, workspace_bytes: int) -> lr_ws_layout:
    arr = (lr_view * len(views))(*views)
    out = lr_ws_layout()
    _check(ctx, load().lr_workspace_layout(ctx, len(views), arr, workspace_bytes, ctypes.byref(out)),
           "lr_workspace_layout")
    return out


def lr_get_stats(ctx, raise_on_error: bool = True) -> lr_stats:
    st = lr_stats()
    status = load().lr_get_stats(ctx, ctypes.byref(st))
    if raise_on_error:
        _check(ctx, status, "lr_get_stats")
    return st


def lr_last_error(ctx) -> str:
    return (load().lr_last_error(ctx) or b"").decode(errors="replace")


def lr_server_start(ctx, config: lr_server_config):
    _check(ctx, load().lr_server_start(ctx, ctypes.byref(config)), "lr_server_start")


def lr_server_stop(ctx):
    _check(ctx, load().lr_server_stop(ctx), "lr_server_stop")


def lr_submit(ctx, view: lr_view) -> int:
    t = ctypes.c_uint64()
    _check(ctx, load().lr_submit(ctx, ctypes.byref(view), ctypes.byref(t)), "lr_submit")
    return t.value


def lr_poll(ctx, ticket: int, timeout_us: int = 0):
    """(call status, request status): call status LR_OK once the request has finished."""
    res = ctypes.c_int(LR_PENDING)
    st = load().lr_poll(ctx, ticket, timeout_us, ctypes.byref(res))
    return st, res.value


def lr_poll_info(ctx, ticket: int, timeout_us: int = 0):
    res = ctypes.c_int(LR_PENDING)
    info = lr_request_info()
    st = load().lr_poll_info(ctx, ticket, timeout_us, ctypes.byref(res), ctypes.byref(info))
    return st, res.value, info


def lr_server_get_stats(ctx) -> lr_server_stats:
    out = lr_server_stats()
    _check(ctx, load().lr_server_get_stats(ctx, ctypes.byref(out)), "lr_server_get_stats")
    return out


def lr_now_ns() -> int:
    return load().lr_now_ns()


def lr_render_noalloc(quads: lr_quads, camera: lr_camera, width: int, height: int, out_rgba: int,
                      device_status: int, stream: int) -> int:
    """Returns the call's lr_status (no exception: callers test the documented codes)."""
    return load().lr_render_noalloc(ctypes.byref(quads), ctypes.byref(camera), width, height,
                                    out_rgba, device_status, stream)


def lr_graph_create(ctx, views, workspace: int, workspace_bytes: int):
    arr = (lr_view * len(views))(*views)
    out = _P()
    _check(ctx, load().lr_graph_create(ctx, len(views), arr, workspace, workspace_bytes, ctypes.byref(out)),
           "lr_graph_create")
    return out


def lr_graph_launch(ctx, graph, views, stream: int):
    arr = None if views is None else (lr_view * len(views))(*views)
    _check(ctx, load().lr_graph_launch(graph, arr, stream), "lr_graph_launch")


def lr_graph_destroy(graph):
    _check(None, load().lr_graph_destroy(graph), "lr_graph_destroy")
