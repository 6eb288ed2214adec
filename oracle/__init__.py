"""CPU oracle for the exact-OIT quad rasteriser (LucidRaster, arXiv 2405.13364).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package; the product library never does, and the two
share no code. The arithmetic lives in ``lr_oracle.c`` (plain C, built with
``-ffp-contract=off`` so that every fp32 operation is rounded separately); this module
only builds it with gcc and marshals numpy arrays through ctypes.

Functions (each follows the definition stated in ``lr_oracle.c``):
  setup(scene)                 per-quad cull status, snapped X/Y, q = 1/w, pixel AABB
  render(scene)                fp32 image, per-pixel fragment count and coverage hash,
                               8-bit image, the fp64 composite of the same fragment order
  render_msaa(scene, offsets)  multisampled image: the mean of the exact images of several
                               sample positions per pixel (offsets from the centre)
  render_pixels(scene, xs, ys) the same quantities for selected pixels only
  render_threshold(scene, t)   the opt-in lossy alpha-threshold composite (front to back,
                               a fragment blended only while transmittance > t)
  render64(scene, colors64)    fp64 forward (flat colours) used for finite differences
Scenes with lit colours (color_mode 2, [V][8] = RGBA, normal, unused) carry their light as
scene.light = (x, y, z toward the light, ambient).
  backward(scene, grad_out)    fp64 gradient w.r.t. flat per-quad RGBA (Sec. 2 blending,
                               differentiated)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblr_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS_NAMES = ["visible", "bad_index", "nonfinite", "depth", "guard", "degenerate", "no_pixel"]


class _Scene(ctypes.Structure):
    _fields_ = [
        ("positions", ctypes.c_void_p), ("num_vertices", ctypes.c_int64),
        ("indices", ctypes.c_void_p), ("num_quads", ctypes.c_int64),
        ("colors", ctypes.c_void_p), ("color_mode", ctypes.c_int32),
        ("view_proj", ctypes.c_void_p), ("near_z", ctypes.c_float), ("far_z", ctypes.c_float),
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("sample_x", ctypes.c_int32), ("sample_y", ctypes.c_int32),
        ("light", ctypes.c_float * 4),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [("quads_by_status", ctypes.c_int64 * 8), ("fragments", ctypes.c_int64),
                ("max_depth", ctypes.c_int64), ("key_ties", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile lr_oracle.c with gcc into oracle/_build/liblr_oracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    P = ctypes.c_void_p
    lib.or_setup.argtypes = [ctypes.POINTER(_Scene), P, P, P, P, P]
    lib.or_render.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, P, P, P, P, P,
                              ctypes.POINTER(_Stats)]
    lib.or_render64.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, P, P]
    lib.or_render_threshold.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, ctypes.c_float,
                                        P, P, P, P]
    lib.or_backward.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, P, P, P]
    lib.or_render_pixels.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int, ctypes.c_int64,
                                     P, P, P, P, P]
    lib.or_num_threads.argtypes = [ctypes.c_int]
    lib.or_pixel_fragments.argtypes = [ctypes.POINTER(_Scene), ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int64, P, P, P, P]
    lib.or_pixel_fragments.restype = ctypes.c_int64
    for f in (lib.or_setup, lib.or_render, lib.or_render64, lib.or_render_threshold, lib.or_backward,
              lib.or_render_pixels, lib.or_num_threads):
        f.restype = ctypes.c_int
    return lib


def build_variant(source_text: str, out_dir: str) -> str:
    """Compile a modified copy of the oracle source (used by tests that plant mistakes
    in the oracle to show that the pins catch them)."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "variant.c")
    lib = os.path.join(out_dir, "libvariant.so")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-pthread", src, "-o", lib, "-lm"], check=True)
    return lib


def use_library(path):
    """Route every oracle call through the library at path (None: the real oracle)."""
    global _lib
    with _lock:
        _lib = None if path is None else _bind(ctypes.CDLL(path))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = _bind(ctypes.CDLL(build()))
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p).value


class _Bound:
    """Keeps contiguous copies alive while the C call runs."""

    def __init__(self, scene, colors=None, sample=(128, 128)):
        self.pos = np.ascontiguousarray(scene.positions, np.float32)
        self.idx = None if scene.indices is None else np.ascontiguousarray(scene.indices, np.uint32)
        self.col = np.ascontiguousarray(scene.colors if colors is None else colors, np.float32)
        self.m = np.ascontiguousarray(scene.view_proj, np.float32).reshape(16)
        q = self.idx.shape[0] if self.idx is not None else self.pos.shape[0] // 4
        self.s = _Scene(_ptr(self.pos), self.pos.shape[0], _ptr(self.idx), q, _ptr(self.col),
                        int(scene.color_mode), _ptr(self.m), float(scene.near), float(scene.far),
                        int(scene.width), int(scene.height), int(sample[0]), int(sample[1]),
                        (ctypes.c_float * 4)(*(getattr(scene, "light", None) or (0.0, 0.0, 0.0, 0.0))))
        self.num_quads = q


def num_threads(n: int = 0) -> int:
    return _load().or_num_threads(n)


def setup(scene):
    lib = _load()
    b = _Bound(scene)
    q = b.num_quads
    status = np.zeros(q, np.int32)
    X = np.zeros((q, 4), np.int32)
    Y = np.zeros((q, 4), np.int32)
    qq = np.zeros((q, 4), np.float32)
    bbox = np.zeros((q, 4), np.int32)
    lib.or_setup(ctypes.byref(b.s), _ptr(status), _ptr(X), _ptr(Y), _ptr(qq), _ptr(bbox))
    return dict(status=status, X=X, Y=Y, q=qq, bbox=bbox)


def render(scene, nthreads: int = 0, want64: bool = False, sample=(128, 128)):
    """sample: the position in each pixel, in 1/256 px from its top-left corner, whose
    coverage makes the image ((128, 128): the pixel centre)."""
    lib = _load()
    b = _Bound(scene, sample=sample)
    H, W = scene.height, scene.width
    rgba = np.zeros((H, W, 4), np.float32)
    count = np.zeros((H, W), np.uint32)
    hsh = np.zeros((H, W), np.uint64)
    rgba8 = np.zeros((H, W, 4), np.uint8)
    rgba64 = np.zeros((H, W, 4), np.float64) if want64 else None
    st = _Stats()
    rc = lib.or_render(ctypes.byref(b.s), nthreads, _ptr(rgba), _ptr(count), _ptr(hsh),
                       _ptr(rgba8), _ptr(rgba64), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"oracle render failed ({rc})")
    stats = dict(fragments=st.fragments, max_depth=st.max_depth, key_ties=st.key_ties,
                 **{STATUS_NAMES[i]: st.quads_by_status[i] for i in range(len(STATUS_NAMES))})
    out = dict(rgba=rgba, count=count, hash=hsh, rgba8=rgba8, stats=stats)
    if want64:
        out["rgba64"] = rgba64
    return out


# Sample offsets from the pixel centre, in 1/256 px (x right, y down). 4 samples: a grid
# rotated so that each sample has its own row and column, offsets (+-1/8, +-3/8) px. 16
# samples: one per row and column of a 16 x 16 sub-grid (cells 1/16 px), the column of row
# i being (5 i + 3) mod 16.
MSAA_OFFSETS = {
    4: [(-32, -96), (96, -32), (-96, 32), (32, 96)],
    16: [(16 * ((5 * i + 3) % 16) - 120, 16 * i - 120) for i in range(16)],
}


def render_msaa(scene, offsets=4, nthreads: int = 0):
    """Multisampled exact OIT: for every sample offset (dx, dy) the exact image with
    coverage, depth and colour taken at (256 px + 128 + dx, 256 py + 128 + dy), then the
    per-pixel mean (fp32 sum in sample order, divided by the sample count). offsets: a
    list of (dx, dy) or a sample count with a default pattern (MSAA_OFFSETS)."""
    if isinstance(offsets, int):
        offsets = MSAA_OFFSETS[offsets]
    acc = None
    samples = []
    for dx, dy in offsets:
        img = render(scene, nthreads, sample=(128 + dx, 128 + dy))["rgba"]
        samples.append(img)
        acc = img.copy() if acc is None else (acc + img).astype(np.float32)
    return (acc / np.float32(len(offsets))).astype(np.float32), samples


def render_pixels(scene, xs, ys, nthreads: int = 0):
    lib = _load()
    b = _Bound(scene)
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    n = xs.shape[0]
    rgba = np.zeros((n, 4), np.float32)
    count = np.zeros(n, np.uint32)
    hsh = np.zeros(n, np.uint64)
    lib.or_render_pixels(ctypes.byref(b.s), nthreads, n, _ptr(xs), _ptr(ys), _ptr(rgba),
                         _ptr(count), _ptr(hsh))
    return dict(rgba=rgba, count=count, hash=hsh)


def pixel_fragments(scene, px: int, py: int, cap: int = 4096):
    """Sorted (back to front) fragments of one pixel: key, quad, triangle, rgba."""
    lib = _load()
    b = _Bound(scene)
    key = np.zeros(cap, np.float32)
    quad = np.zeros(cap, np.uint32)
    tri = np.zeros(cap, np.uint32)
    rgba = np.zeros((cap, 4), np.float32)
    n = lib.or_pixel_fragments(ctypes.byref(b.s), px, py, cap, _ptr(key), _ptr(quad), _ptr(tri),
                               _ptr(rgba))
    n = min(n, cap)
    return dict(key=key[:n], quad=quad[:n], tri=tri[:n], rgba=rgba[:n])


def render_threshold(scene, t_min: float = 1.0 / 128.0, nthreads: int = 0):
    """Alpha-threshold composite: rgba, per-pixel fragments blended (nblend), fragment
    count, and the relative distance of T to t_min at the stop tests (margin)."""
    lib = _load()
    b = _Bound(scene)
    H, W = scene.height, scene.width
    rgba = np.zeros((H, W, 4), np.float32)
    nblend = np.zeros((H, W), np.uint32)
    count = np.zeros((H, W), np.uint32)
    margin = np.zeros((H, W), np.float32)
    rc = lib.or_render_threshold(ctypes.byref(b.s), nthreads, float(t_min), _ptr(rgba),
                                 _ptr(nblend), _ptr(count), _ptr(margin))
    if rc != 0:
        raise RuntimeError(f"oracle render_threshold failed ({rc})")
    return dict(rgba=rgba, nblend=nblend, count=count, margin=margin)


def render64(scene, colors64=None, nthreads: int = 0):
    lib = _load()
    b = _Bound(scene)
    c64 = None if colors64 is None else np.ascontiguousarray(colors64, np.float64)
    out = np.zeros((scene.height, scene.width, 4), np.float64)
    rc = lib.or_render64(ctypes.byref(b.s), nthreads, _ptr(c64), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle render64 failed ({rc})")
    return out


def backward(scene, grad_out, colors64=None, nthreads: int = 0):
    lib = _load()
    b = _Bound(scene)
    g = np.ascontiguousarray(grad_out, np.float64)
    c64 = None if colors64 is None else np.ascontiguousarray(colors64, np.float64)
    out = np.zeros((b.num_quads, 4), np.float64)
    rc = lib.or_backward(ctypes.byref(b.s), nthreads, _ptr(c64), _ptr(g), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"oracle backward failed ({rc})")
    return out


def loss_l2(rgba, target_rgba):
    """L = sum over pixels and RGB channels of (C - T)^2 (the squared L2 distance)."""
    d = rgba[..., :3].astype(np.float64) - target_rgba[..., :3].astype(np.float64)
    return float(np.sum(d * d))


def loss_l2_grad(rgba, target_rgba):
    """dL/d(C, A): 2 (C - T) on RGB, 0 on alpha."""
    g = np.zeros(rgba.shape, np.float64)
    g[..., :3] = 2.0 * (rgba[..., :3].astype(np.float64) - target_rgba[..., :3].astype(np.float64))
    return g
