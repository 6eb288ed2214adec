"""Brute-force restatement of the oracle for tiny images (TEST INFRASTRUCTURE ONLY).

A second, independent enumeration of the same definition: for every pixel, loop over
every quad and both triangles, evaluate the edge functions with unbounded Python
integers, compute the depth key with numpy float32 scalars (one IEEE rounding per
operation), sort the fragment tuples with ``sorted`` and composite back to front.
It shares no code with ``lr_oracle.c``; it exists to catch enumeration mistakes there
(bounding boxes, band limits, index arithmetic, 64-bit overflow) on 16x16 images.
"""
from __future__ import annotations

import numpy as np

f32 = np.float32
GUARD = f32(16384.0)


def _row(m, r, x, y, z):
    a = f32(m[r, 0]) * x
    b = f32(m[r, 1]) * y
    s = f32(a + b)
    c = f32(m[r, 2]) * z
    s = f32(s + c)
    return f32(s + f32(m[r, 3]))


def _snap(v):
    # round half to even on the exactly representable product v*256
    return int(np.rint(f32(v * f32(256.0))))


def _owned(dx, dy):
    return dy < 0 or (dy == 0 and dx > 0)


def _mix(x):
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def _quad_vertices(scene, j):
    if scene.indices is not None:
        return [int(v) for v in scene.indices[j]]
    return [4 * j + k for k in range(4)]


def snapped_quads(scene):
    """Per quad: None if culled, else (X[4], Y[4], q[4], vertex ids)."""
    m = np.asarray(scene.view_proj, np.float32)
    W, H = scene.width, scene.height
    out = []
    for j in range(scene.num_quads):
        vids = _quad_vertices(scene, j)
        ok = True
        X, Y, Q = [], [], []
        for v in vids:
            if v >= scene.num_vertices:
                ok = False
                break
            x, y, z = (f32(c) for c in scene.positions[v])
            with np.errstate(all="ignore"):
                cx, cy, w = _row(m, 0, x, y, z), _row(m, 1, x, y, z), _row(m, 3, x, y, z)
                if not (np.isfinite(cx) and np.isfinite(cy) and np.isfinite(w)):
                    ok = False
                    break
                if not (w >= f32(scene.near) and w <= f32(scene.far)):
                    ok = False
                    break
                sx = f32(f32(f32(cx / w) + f32(1.0)) * f32(f32(0.5) * f32(W)))
                sy = f32(f32(f32(1.0) - f32(cy / w)) * f32(f32(0.5) * f32(H)))
            if not (abs(sx) <= GUARD and abs(sy) <= GUARD):
                ok = False
                break
            X.append(_snap(sx))
            Y.append(_snap(sy))
            Q.append(f32(f32(1.0) / w))
        out.append((X, Y, Q, vids) if ok else None)
    return out


def render(scene, sample=(128, 128)):
    """Returns (rgba f32[H][W][4], count u32[H][W], hash u64[H][W]); sample is the position
    in each pixel (1/256 px from its top-left corner) whose coverage is tested."""
    W, H = scene.width, scene.height
    quads = snapped_quads(scene)
    rgba = np.zeros((H, W, 4), np.float32)
    count = np.zeros((H, W), np.uint32)
    hsh = np.zeros((H, W), np.uint64)
    cols = np.asarray(scene.colors, np.float32)
    for py in range(H):
        for px in range(W):
            Px, Py = 256 * px + sample[0], 256 * py + sample[1]
            frags = []
            for j, qd in enumerate(quads):
                if qd is None:
                    continue
                X, Y, Q, vids = qd
                for t, (a, b, c) in enumerate(((0, 1, 2), (0, 2, 3))):
                    A = (X[b] - X[a]) * (Y[c] - Y[a]) - (Y[b] - Y[a]) * (X[c] - X[a])
                    if A == 0:
                        continue
                    if A < 0:
                        b, c = c, b
                        A = -A
                    V = (a, b, c)

                    def E(u, v):
                        return (X[v] - X[u]) * (Py - Y[u]) - (Y[v] - Y[u]) * (Px - X[u])

                    es = (E(V[1], V[2]), E(V[2], V[0]), E(V[0], V[1]))
                    own = (_owned(X[V[2]] - X[V[1]], Y[V[2]] - Y[V[1]]),
                           _owned(X[V[0]] - X[V[2]], Y[V[0]] - Y[V[2]]),
                           _owned(X[V[1]] - X[V[0]], Y[V[1]] - Y[V[0]]))
                    if not all(e > 0 or (e == 0 and o) for e, o in zip(es, own)):
                        continue
                    inv = f32(f32(1.0) / f32(A))
                    l1 = f32(f32(es[1]) * inv)
                    l2 = f32(f32(es[2]) * inv)
                    q0, q1, q2 = Q[V[0]], Q[V[1]], Q[V[2]]
                    key = f32(q0 + f32(f32(l1 * f32(q1 - q0)) + f32(l2 * f32(q2 - q0))))
                    if scene.color_mode == 0:
                        col = cols[j]
                    else:
                        ls = [es[k] / A for k in range(3)]
                        wk = [ls[k] * float(Q[V[k]]) for k in range(3)]
                        ws = sum(wk)
                        col = np.array([sum(wk[k] * float(cols[vids[V[k]], ch]) for k in range(3)) / ws
                                        for ch in range(4)], np.float32)
                    frags.append((float(key), j, t, col))
            frags.sort(key=lambda f: (f[0], f[1], f[2]))
            C = [f32(0.0)] * 3
            Aout = f32(0.0)
            h = 0
            for key, j, t, col in frags:
                a = f32(col[3])
                om = f32(f32(1.0) - a)
                C = [f32(f32(a * f32(col[ch])) + f32(om * C[ch])) for ch in range(3)]
                Aout = f32(a + f32(om * Aout))
                h = (h + _mix(2 * j + t)) & ((1 << 64) - 1)
            rgba[py, px] = [C[0], C[1], C[2], Aout]
            count[py, px] = len(frags)
            hsh[py, px] = h
    return rgba, count, hsh

