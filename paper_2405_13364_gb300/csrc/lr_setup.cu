// lr_setup.cu -- Stage 1 of the pipeline: quad setup (Sec. 2, "Stage 1: quad setup").
//
// One thread per input quad. Phase 1 of the paper (cull) and Phase 2 (pre-compute and
// store) are fused: the thread loads its four vertex indices and positions with
// vectorised, coalesced loads, transforms them, decides visibility and writes the
// per-quad records that binning and rasterisation read. Records are stored at the quad's
// own index (no compaction); culled quads get an "invisible" rectangle so later stages
// skip them with one 8-byte load.
//
// Exact arithmetic: every fp32 operation that decides coverage or depth order uses the
// explicitly rounded intrinsics (__fmul_rn, __fadd_rn, __frcp_rn), which are never fused
// into multiply-adds, and the two quotients by w are correctly rounded (div_rn_by), so the
// results are bit-identical to any IEEE implementation that evaluates the same operations
// in the same order:
//   c_r  = ((M[r][0] x + M[r][1] y) + M[r][2] z) + M[r][3]        (rows x, y, w)
//   sx   = ((cx / w) + 1) * (W / 2),  sy = (1 - (cy / w)) * (H / 2)
//   X    = rint(sx * 256) (8 fractional bits, round half to even),  q = 1 / w
// and a quad is culled whole if any vertex is non-finite, has w outside [near, far] or
// lands outside the +-16384 px guard band, if both triangles (v0 v1 v2), (v0 v2 v3) have
// zero doubled area, or if its pixel-centre AABB clipped to the screen is empty (Sec. 2,
// Stage 1, Phase 1: culling of quads that fall between sample positions).
#include "lr_common.cuh"

namespace lr {

// Zeroes the control block and the bin counters and writes the first views' descriptors.
// Launched with block 0 covering the whole control block, so the final store of refs_cap is
// ordered after its zeroing.
__global__ void k_init(Ws ws, unsigned long long refs_cap, ViewChunk views, ViewDev* views_dst) {
  pdl_begin();
  if (blockIdx.x == 0 && threadIdx.x < views.count) views_dst[views.first + threadIdx.x] = views.v[threadIdx.x];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (i < (long long)(sizeof(Ctrl) / 4)) reinterpret_cast<uint32_t*>(ws.ctrl)[i] = 0u;
  for (long long b = i; b < ws.total_bins; b += stride) ws.bin_count[b] = 0u;
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) ws.ctrl->refs_cap = refs_cap;
}

__device__ __forceinline__ float row_dot(const float* m, float x, float y, float z) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[0], x), __fmul_rn(m[1], y)), __fmul_rn(m[2], z)),
                   m[3]);
}

__global__ __launch_bounds__(256) void k_setup(Ws ws) {
  pdl_begin();
  const long long g = blockIdx.x * 256LL + threadIdx.x;
  const bool active = g < ws.total_quads;
  uint32_t reason = kVisible;
  if (active) {
    const int v = view_of_quad(ws.views, ws.n_views, g);
    const ViewDev& V = ws.views[v];
    const long long j = g - V.quad_base;
    // ---- load vertex indices and positions ------------------------------------------
    long long vid[4];
    if (V.idx) {
      const uint4 t = __ldg(reinterpret_cast<const uint4*>(V.idx) + j);
      vid[0] = t.x; vid[1] = t.y; vid[2] = t.z; vid[3] = t.w;
    } else {
      for (int k = 0; k < 4; ++k) vid[k] = 4 * j + k;
    }
    float px[4], py[4], pz[4];
    bool bad = false;
    if (!V.idx && 4 * j + 3 < V.num_vertices) {
      // 48 contiguous bytes per quad: three 16-byte loads
      const float4* p4 = reinterpret_cast<const float4*>(V.pos) + 3 * j;
      const float4 a = __ldg(p4), b = __ldg(p4 + 1), c = __ldg(p4 + 2);
      px[0] = a.x; py[0] = a.y; pz[0] = a.z;
      px[1] = a.w; py[1] = b.x; pz[1] = b.y;
      px[2] = b.z; py[2] = b.w; pz[2] = c.x;
      px[3] = c.y; py[3] = c.z; pz[3] = c.w;
    } else {
      for (int k = 0; k < 4; ++k) {
        if (vid[k] >= V.num_vertices) { bad = true; px[k] = py[k] = pz[k] = 0.f; continue; }
        const float* p = V.pos + 3 * vid[k];
        px[k] = __ldg(p); py[k] = __ldg(p + 1); pz[k] = __ldg(p + 2);
      }
    }
    // ---- transform, classify, snap ----------------------------------------------------
    int X[4] = {0, 0, 0, 0}, Y[4] = {0, 0, 0, 0};
    float q[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t worst = bad ? (uint32_t)kBadIndex : (uint32_t)kVisible;
    for (int k = 0; k < 4; ++k) {
      if (vid[k] >= V.num_vertices) continue;
      const float cx = row_dot(V.m + 0, px[k], py[k], pz[k]);
      const float cy = row_dot(V.m + 4, px[k], py[k], pz[k]);
      const float w = row_dot(V.m + 8, px[k], py[k], pz[k]);
      uint32_t why = kVisible;
      if (!isfinite(cx) || !isfinite(cy) || !isfinite(w)) {
        why = kNonFinite;
      } else if (!(w >= V.near_z && w <= V.far_z)) {
        why = kDepth;
      } else {
        // q = 1/w correctly rounded; cx / w and cy / w from it by a correction that gives
        // the correctly rounded quotient (div_rn_by)
        const float qk = __frcp_rn(w);
        const float sx = __fmul_rn(__fadd_rn(div_rn_by(cx, w, qk), 1.0f), V.half_w);
        const float sy = __fmul_rn(__fsub_rn(1.0f, div_rn_by(cy, w, qk)), V.half_h);
        if (!(fabsf(sx) <= kGuardPx && fabsf(sy) <= kGuardPx)) {
          why = kGuard;
        } else {
          // (minus the sample offset of a multisampled view: edge values, the depth key and
          // the colour weights are differences of vertex positions and the tested point, so
          // moving the vertices by -d tests the point centre + d exactly)
          X[k] = __float2int_rn(__fmul_rn(sx, 256.0f)) - V.sub_x;
          Y[k] = __float2int_rn(__fmul_rn(sy, 256.0f)) - V.sub_y;
          q[k] = qk;
        }
      }
      if (why != kVisible && (worst == kVisible || why < worst)) worst = why;
    }
    uint32_t info = 0;
    float rep = 0.f;
    float2 inv = make_float2(0.f, 0.f);
    uint2 rect = make_uint2(kRectInvisible, kRectInvisible);
    if (worst == kVisible) {
      const long long a0 = area2(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
      const long long a1 = area2(X[0], Y[0], X[2], Y[2], X[3], Y[3]);
      if (a0 == 0 && a1 == 0) {
        worst = kDegenerate;
      } else {
        info |= (a0 != 0 ? kInfoTri0 : 0u) | (a1 != 0 ? kInfoTri1 : 0u);
        // per-triangle constants that every half-block would otherwise recompute: the
        // orientation, 1/area of the depth interpolation (Sec. 2, "Stage 3"), and whether
        // 32-bit edge arithmetic is exact wherever the triangle is rasterised. A half-block
        // touching the triangle's pixel box holds pixel centres within 7 px (x) and 3 px (y)
        // of the vertex box, so |E| <= Wx (Wy + 3*256) + Wy (Wx + 7*256) + 1 there.
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          long long A = t ? a1 : a0;
          if (A == 0) continue;
          if (A < 0) {
            info |= kInfoSwap0 << t;
            A = -A;
          }
          const float it = __frcp_rn(__ll2float_rn(A));
          if (t) inv.y = it; else inv.x = it;
          const int xb = t ? X[2] : X[1], yb = t ? Y[2] : Y[1], xc = t ? X[3] : X[2], yc = t ? Y[3] : Y[2];
          // (vertex boxes lie within the guard band, so the extents fit 32 bits; below 2^15
          // each the bound's two products and their sum fit an unsigned 32-bit word)
          const uint32_t wx = (uint32_t)(max(X[0], max(xb, xc)) - min(X[0], min(xb, xc)));
          const uint32_t wy = (uint32_t)(max(Y[0], max(yb, yc)) - min(Y[0], min(yb, yc)));
          if (wx < 32768u && wy < 32768u && wx * (wy + 3u * 256u) + wy * (wx + 7u * 256u) + 1u < (1u << 30))
            info |= kInfoSmall0 << t;
        }
        const int xmin = min(min(X[0], X[1]), min(X[2], X[3]));
        const int xmax = max(max(X[0], X[1]), max(X[2], X[3]));
        const int ymin = min(min(Y[0], Y[1]), min(Y[2], Y[3]));
        const int ymax = max(max(Y[0], Y[1]), max(Y[2], Y[3]));
        const int px0 = max(ceil_div256((long long)xmin - 128), 0);
        const int px1 = min(floor_div256((long long)xmax - 128), V.width - 1);
        const int py0 = max(ceil_div256((long long)ymin - 128), 0);
        const int py1 = min(floor_div256((long long)ymax - 128), V.height - 1);
        if (px0 > px1 || py0 > py1) {
          worst = kNoPixel;
        } else {
          rect = make_uint2((uint32_t)px0 | ((uint32_t)px1 << 16), (uint32_t)py0 | ((uint32_t)py1 << 16));
          const int bw = (px1 >> ws.bin_log2) - (px0 >> ws.bin_log2) + 1;
          const int bh = (py1 >> ws.bin_log2) - (py0 >> ws.bin_log2) + 1;
          if (bw > kSmallBins || bh > kSmallBins) info |= kInfoLarge;
          if (q[0] == q[1] && q[0] == q[2] && q[0] == q[3]) info |= kInfoFlatDepth;
          rep = rep_depth_of(X, Y, q, info, px0, px1, py0, py1);
        }
      }
    }
    if (worst != kVisible) {
      info = 0;
      rect = make_uint2(kRectInvisible, kRectInvisible);
    }
    reason = worst;
    // later stages read the record and the representative depth of visible quads only (a
    // culled quad's invisible rectangle keeps it out of every bin), so culled quads skip them
    if (worst == kVisible) {
      int4* rp = ws.rec + 4 * g;
      rp[0] = make_int4(X[0], Y[0], X[1], Y[1]);
      rp[1] = make_int4(X[2], Y[2], X[3], Y[3]);
      rp[2] = make_int4(__float_as_int(q[0]), __float_as_int(q[1]), __float_as_int(q[2]), __float_as_int(q[3]));
      rp[3] = make_int4(__float_as_int(inv.x), __float_as_int(inv.y), (int)info, 0);
      ws.rec_rep[g] = rep;
    }
    ws.rec_rect[g] = rect;
    ws.rec_info[g] = info | (worst << 8);
    if (bad) set_error(ws.ctrl, LR_ERR_INVALID_ARG);
  }
  // statistics: culled quads per reason, one atomic per reason present in the warp, by its
  // lowest lane (the host derives the visible count, so warps without a culled quad issue
  // no atomic)
  const unsigned culled = __ballot_sync(0xffffffffu, active && reason != kVisible);
  if (culled) {
    const unsigned peers = __match_any_sync(0xffffffffu, active ? reason : kVisible);
    const int lane = threadIdx.x & 31;
    if (((culled >> lane) & 1u) && lane == __ffs(peers) - 1)
      atomicAdd(&ws.ctrl->culled[reason], (unsigned long long)__popc(peers));
  }
}

}  // namespace lr
