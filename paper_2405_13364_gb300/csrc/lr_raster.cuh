// lr_raster.cuh -- Stage 3 of the pipeline, bin rasterisation (Sec. 2, "Stage 3: bin
// rasterization"), with the exact fallback the paper sketches (Sec. 2, "Sample blending").
//
// Work decomposition. Every 32x32 bin is cut into 32 half-blocks of 8x4 pixels (the
// paper's tri-half-block granularity). A half-block is one work item and one warp: lane
// = pixel. Persistent warps take items from a device queue ordered by bin size (largest
// bins first), so high-density bins are spread over many warps instead of one CTA.
//
// Per half-block (all from the bin's reference list, already sorted front to back by
// k_bin_sort -- stage 1 of the two-stage sort, Sec. 2, Stage 3, Phase 2):
//   1. candidates: the half-block's row of the bin's transposed bitmap (written by
//      k_bin_sort: bit j set iff sorted reference j overlaps the half-block) is read with
//      one coalesced load per 1024 references, and its set bits are handed out 32 at a
//      time in sorted order, one candidate quad per lane;
//   2. triangle setup, lane-parallel: for 32 candidate quads, both triangles' integer edge
//      functions at the half-block origin, per-pixel steps, 1/area, depth-plane deltas;
//      a triangle whose edge values stay below 2^30 on the half-block is marked "fast"
//      and evaluated with 32-bit integers, others with exact 64-bit integers; the same
//      lane computes each triangle's 32-pixel coverage mask (top-left rule) row by row;
//   3. coverage, transposed: a 32x32 bit transpose across the warp turns "triangle ->
//      pixels" into "pixel -> triangles", one bit per covering triangle in each lane;
//   4. fragments, per lane in candidate order: the exact depth key of the fragment
//      (interpolated 1/w, identical bit for bit to the oracle's formula) is pushed into a
//      K-slot register sorter (stage 2, the paper's depth filter, Sec. 2, Stage 3,
//      Phase 3, "Sample blending"). When full,
//      the nearest element is evicted and blended front to back. If a fragment arrives
//      that is nearer than the last evicted one, the stream was not in order for this
//      pixel: the pixel is flagged (the paper's misorder detection, same passage) and
//      registered for k_overflow.
// Sort keys are (float bits of key) << 32 | (2 * quad + triangle): distinct per pixel, so
// the per-pixel order is total and the result is unique.
#pragma once

#include "lr_common.cuh"

namespace lr {

constexpr uint32_t kTriValid = 1u, kTriFast = 2u, kTriFlatCol = 4u;   // + corr bits 3..5
// all three vertices at the same 1/w: the depth key is q0 at every pixel (the
// interpolation adds l1 * 0 + l2 * 0 with l1, l2 >= 0)
constexpr uint32_t kTriConstKey = 64u;
// lit colours (LR_COLOR_LIT): the triangle's colour slots also hold its perspective-weighted
// normals, and each fragment's RGB is shaded with the view's light
constexpr uint32_t kTriLit = 128u;
constexpr unsigned long long kSent = ~0ull;
constexpr int kRasterThreads = 256;
#ifndef LR_RASTER_MIN_BLOCKS
// resident CTAs per SM requested from the compiler: 3 caps registers at 80 per thread (24
// warps per SM, a few spills), measured faster than 2 (128 registers) on both the layer
// and the particle workloads; without a bound the compiler takes ~160 and one CTA fits
#define LR_RASTER_MIN_BLOCKS 3
#endif
constexpr int kRasterWarps = kRasterThreads / 32;
constexpr int kOvfThreads = 128;
// alpha threshold (LR_FLAG_ALPHA_THRESHOLD, the paper's opt-in early stop, Sec. 2 "Sample
// blending"): a pixel blends a fragment only while its transmittance is above this, i.e.
// until its accumulated alpha reaches 1 - 1/128
constexpr float kAlphaTMin = 1.0f / 128.0f;
// The fp32 depth key of any fragment of a quad is at most its largest vertex 1/w times
// this: the key is a convex combination of three vertex values evaluated with a handful
// of roundings of relative size 2^-24 each, far inside the 2^-16 margin.
constexpr float kKeyBoundScale = 1.0f + 1.0f / 65536.0f;

// Per (triangle, half-block) record read by the fragment loop, laid out for three 16-byte
// shared-memory loads. Edges 1 (v2->v0) and 2 (v0->v1) give the barycentric numerators
// of the depth key; edge 0 is only needed for coverage, which the masks already hold.
struct __align__(16) TriSm {
  int4 ea;         // e1, e2: edge values E at the half-block's first pixel centre; sx1,
                   // sx2: change per pixel step in x
  int4 eb;         // sy1, sy2: change per pixel step in y; flags; id (2 * quad + triangle)
  float4 kq;       // q0 = 1/w at v0, d1 = q1 - q0, d2 = q2 - q0, inv = 1 / (float)area
  int X[3], Y[3];  // vertices after the orientation fix (64-bit path)
  int pad[2];
};

// dynamic shared memory of k_raster: per warp 64 triangle records, when fragments carry
// colours 3 premultiplied vertex colours per triangle (6 slots with lit colours: also the
// weighted normals), and for the backward 32 gradient slots
__host__ __device__ constexpr int col_slots(bool lit) { return lit ? 6 : 3; }
__host__ __device__ constexpr size_t raster_smem_bytes(bool vtx, bool bwd = false, bool lit = false) {
  return (size_t)kRasterWarps * 64 * sizeof(TriSm) +
         (vtx ? (size_t)kRasterWarps * 64 * col_slots(lit) * sizeof(float4) : 0) +
         (bwd ? (size_t)kRasterWarps * 32 * sizeof(float4) : 0);
}

// exact 64-bit edge values (unbiased) of a triangle at pixel (px, py)
__device__ __forceinline__ void edges64(const TriSm& T, int px, int py, long long e[3]) {
  const long long Px = 256LL * px + 128, Py = 256LL * py + 128;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int u = k == 0 ? 1 : (k == 1 ? 2 : 0);
    const int w = k == 0 ? 2 : (k == 1 ? 0 : 1);
    e[k] = (long long)(T.X[w] - T.X[u]) * (Py - T.Y[u]) - (long long)(T.Y[w] - T.Y[u]) * (Px - T.X[u]);
  }
}

// Builds the per-half-block record of triangle t of a quad; returns false if the triangle
// has zero area or its pixel AABB misses the half-block (BH rows: 4, or 8 for the 8x8
// blocks of k_raster8).
template <int BH = kHbH>
static __device__ __noinline__ bool setup_tri(TriSm& T, const int X[4], const int Y[4], const float qv[4],
                                          uint32_t info, int t, uint32_t jl, int ox, int oy,
                                          int cor[3], int box[4], int le[3], int lsx[3], int lsy[3]) {
  if (!(info & (t ? kInfoTri1 : kInfoTri0))) return false;
  // vertices (v0, v1, v2) of T0 or (v0, v2, v3) of T1, chosen with selects (no indexing)
  int xa = X[0], ya = Y[0];
  int xb = t ? X[2] : X[1], yb = t ? Y[2] : Y[1];
  int xc = t ? X[3] : X[2], yc = t ? Y[3] : Y[2];
  float qa = qv[0], qb = t ? qv[2] : qv[1], qc = t ? qv[3] : qv[2];
  int ib = t ? 2 : 1, ic = t ? 3 : 2;
  long long A = area2(xa, ya, xb, yb, xc, yc);
  if (A < 0) {   // orientation fix: swap v1 and v2
    int ti = xb; xb = xc; xc = ti;
    ti = yb; yb = yc; yc = ti;
    const float tq = qb; qb = qc; qc = tq;
    ti = ib; ib = ic; ic = ti;
    A = -A;
  }
  const int xmin = min(xa, min(xb, xc)), xmax = max(xa, max(xb, xc));
  const int ymin = min(ya, min(yb, yc)), ymax = max(ya, max(yb, yc));
  const int bx0 = ceil_div256((long long)xmin - 128), bx1 = floor_div256((long long)xmax - 128);
  const int by0 = ceil_div256((long long)ymin - 128), by1 = floor_div256((long long)ymax - 128);
  if (bx0 > ox + kHbW - 1 || bx1 < ox || by0 > oy + BH - 1 || by1 < oy) return false;
  box[0] = max(bx0 - ox, 0);
  box[1] = min(bx1 - ox, kHbW - 1);
  box[2] = max(by0 - oy, 0);
  box[3] = min(by1 - oy, BH - 1);
  cor[0] = 0; cor[1] = ib; cor[2] = ic;
  T.X[0] = xa; T.X[1] = xb; T.X[2] = xc;
  T.Y[0] = ya; T.Y[1] = yb; T.Y[2] = yc;
  T.kq = make_float4(qa, __fsub_rn(qb, qa), __fsub_rn(qc, qa), __fdiv_rn(1.0f, __ll2float_rn(A)));
  uint32_t flags = kTriValid | ((qb == qa && qc == qa) ? kTriConstKey : 0u);
  bool fast = true;
  const long long P0x = 256LL * ox + 128, P0y = 256LL * oy + 128;
  const long long lim = 1LL << 30;
  // edges v1->v2, v2->v0, v0->v1
  const int ux[3] = {xb, xc, xa}, uy[3] = {yb, yc, ya}, wx[3] = {xc, xa, xb}, wy[3] = {yc, ya, yb};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const long long dx = (long long)wx[k] - ux[k], dy = (long long)wy[k] - uy[k];
    const bool owned = dy < 0 || (dy == 0 && dx > 0);
    const long long e0 = dx * (P0y - uy[k]) - dy * (P0x - ux[k]) + (owned ? 0 : -1);
    const long long sx = -256 * dy, sy = 256 * dx;
    const long long c1 = e0 + (kHbW - 1) * sx, c2 = e0 + (BH - 1) * sy, c3 = c1 + (BH - 1) * sy;
    fast &= (e0 > -lim && e0 < lim && c1 > -lim && c1 < lim && c2 > -lim && c2 < lim && c3 > -lim && c3 < lim);
    le[k] = (int)e0;
    lsx[k] = (int)sx;
    lsy[k] = (int)sy;
    if (!owned) flags |= 1u << (3 + k);
  }
  if (fast) flags |= kTriFast;
  // the key's edge values unbiased (the masks use the biased ones in le)
  T.ea = make_int4((int)((uint32_t)le[1] + ((flags >> 4) & 1u)), (int)((uint32_t)le[2] + ((flags >> 5) & 1u)), lsx[1],
                   lsx[2]);
  T.eb = make_int4(lsy[1], lsy[2], (int)flags, (int)(2u * jl + (uint32_t)t));
  return true;
}

// setup_tri for a triangle that k_setup marked small (kInfoSmall0 << t): the orientation
// and 1/area come precomputed, and every edge value at the pixel centres of the box's rows,
// up to 7 pixels to either side of the box, fits in 32 bits, so the whole set-up is 32-bit
// integer arithmetic (a block row outside the box is masked off, whatever its values).
template <int BH = kHbH>
__device__ __forceinline__ bool setup_tri_small(TriSm& T, const int X[4], const int Y[4], const float qv[4],
                                                float inv, uint32_t info, int t, uint32_t jl, int ox, int oy,
                                                int cor[3], int box[4], int le[3], int lsx[3], int lsy[3]) {
  if (!(info & (t ? kInfoTri1 : kInfoTri0))) return false;
  int xa = X[0], ya = Y[0];
  int xb = t ? X[2] : X[1], yb = t ? Y[2] : Y[1];
  int xc = t ? X[3] : X[2], yc = t ? Y[3] : Y[2];
  float qa = qv[0], qb = t ? qv[2] : qv[1], qc = t ? qv[3] : qv[2];
  int ib = t ? 2 : 1, ic = t ? 3 : 2;
  if (info & (kInfoSwap0 << t)) {
    int ti = xb; xb = xc; xc = ti;
    ti = yb; yb = yc; yc = ti;
    const float tq = qb; qb = qc; qc = tq;
    ti = ib; ib = ic; ic = ti;
  }
  // pixel-centre box: ceil((min - 128) / 256) .. floor((max - 128) / 256)
  const int bx0 = (min(xa, min(xb, xc)) + 127) >> 8, bx1 = (max(xa, max(xb, xc)) - 128) >> 8;
  const int by0 = (min(ya, min(yb, yc)) + 127) >> 8, by1 = (max(ya, max(yb, yc)) - 128) >> 8;
  if (bx0 > ox + kHbW - 1 || bx1 < ox || by0 > oy + BH - 1 || by1 < oy) return false;
  box[0] = max(bx0 - ox, 0);
  box[1] = min(bx1 - ox, kHbW - 1);
  box[2] = max(by0 - oy, 0);
  box[3] = min(by1 - oy, BH - 1);
  cor[0] = 0; cor[1] = ib; cor[2] = ic;
  T.kq = make_float4(qa, __fsub_rn(qb, qa), __fsub_rn(qc, qa), inv);
  uint32_t flags = kTriValid | kTriFast | ((qb == qa && qc == qa) ? kTriConstKey : 0u);
  const int P0x = 256 * ox + 128, P0y = 256 * oy + 128;
  const int ux[3] = {xb, xc, xa}, uy[3] = {yb, yc, ya}, wx[3] = {xc, xa, xb}, wy[3] = {yc, ya, yb};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int dx = wx[k] - ux[k], dy = wy[k] - uy[k];
    const bool owned = dy < 0 || (dy == 0 && dx > 0);
    le[k] = (int)((uint32_t)dx * (uint32_t)(P0y - uy[k]) - (uint32_t)dy * (uint32_t)(P0x - ux[k])) - (owned ? 0 : 1);
    lsx[k] = -256 * dy;
    lsy[k] = 256 * dx;
    if (!owned) flags |= 1u << (3 + k);
  }
  // the key's edge values unbiased (the masks use the biased ones in le)
  T.ea = make_int4((int)((uint32_t)le[1] + ((flags >> 4) & 1u)), (int)((uint32_t)le[2] + ((flags >> 5) & 1u)), lsx[1],
                   lsx[2]);
  T.eb = make_int4(lsy[1], lsy[2], (int)flags, (int)(2u * jl + (uint32_t)t));
  return true;
}

// Backward of the front-to-back composite for one pixel (flat per-quad RGBA). With
// C = sum_i T_i a_i c_i, T_i = prod_{k<i} (1 - a_k), A = 1 - prod (1 - a_k):
//   dC/dc_i = T_i a_i,   dC/da_i = T_i c_i - S_i / (1 - a_i),   dA/da_i = T_final / (1 - a_i)
// where S_i = C_final - (C accumulated through fragment i) is the colour contributed by the
// fragments behind i. C_final, T_final come from the forward image; the running sums are
// recomputed with the forward's operations in the forward's order.
struct GradPixel {
  float gr, gg, gb, ga;      // dL/d(R, G, B, A) of the pixel
  float fr, fg, fb, fT;      // forward colour and transmittance
  float* grad;               // f32[Q][4] of the view
  float4* agg;               // this warp's 32 shared-memory slots for combining lanes' gradients
};

// Columns lx in [0, 8) of one half-block row where an edge is non-negative, as an 8-bit
// mask, given the edge value r at lx = 0 and its step sx per column. The edge is linear in
// lx, so the failing columns form a prefix (sx >= 0) or a suffix (sx < 0); mirroring the
// row turns the suffix into a prefix, whose length is found by a 4-step binary search on
// exact 32-bit edge values (every value evaluated is a pixel centre of the half-block).
__device__ __forceinline__ uint32_t row_cover(int r, int sx) {
  const bool neg = sx < 0;
  const uint32_t g0 = neg ? (uint32_t)r + 7u * (uint32_t)sx : (uint32_t)r;
  const uint32_t sa = neg ? 0u - (uint32_t)sx : (uint32_t)sx;
  int cnt = ((int)(g0 + 3u * sa) < 0) ? 4 : 0;
  cnt += ((int)(g0 + (uint32_t)(cnt + 1) * sa) < 0) ? 2 : 0;
  cnt += ((int)(g0 + (uint32_t)cnt * sa) < 0) ? 1 : 0;
  cnt += (cnt == 7 && (int)(g0 + 7u * sa) < 0) ? 1 : 0;
  return neg ? (0xFFu >> cnt) : ((0xFFu << cnt) & 0xFFu);
}

// Coverage of the half-block's 32 pixel centres (bit ly * 8 + lx) by a "fast" triangle:
// per row the intersection of the three edges' covered columns, limited to the triangle's
// pixel bounding box.
__device__ __forceinline__ uint32_t tri_mask_fast(const int e[3], const int sx[3], const int sy[3],
                                                  const int box[4]) {
  uint32_t mask = 0;
  const uint32_t cols = ((2u << box[1]) - 1u) & ~((1u << box[0]) - 1u);
#pragma unroll
  for (int ly = 0; ly < kHbH; ++ly) {
    uint32_t row = (ly >= box[2] && ly <= box[3]) ? cols : 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      row &= row_cover((int)((uint32_t)e[k] + (uint32_t)ly * (uint32_t)sy[k]), sx[k]);
    mask |= row << (ly * kHbW);
  }
  return mask;
}

// The same for a triangle of a quad whose diagonal's coverage is given: d = the half-block's
// mask of the diagonal in this triangle's direction; only the other two edges (e0, e1, with
// their steps) are evaluated.
__device__ __forceinline__ uint32_t tri_mask_two(int e0, int sx0, int sy0, int e1, int sx1, int sy1, uint32_t d,
                                                 const int box[4]) {
  uint32_t mask = 0;
  const uint32_t cols = ((2u << box[1]) - 1u) & ~((1u << box[0]) - 1u);
#pragma unroll
  for (int ly = 0; ly < kHbH; ++ly) {
    uint32_t row = (ly >= box[2] && ly <= box[3]) ? cols : 0u;
    row &= row_cover((int)((uint32_t)e0 + (uint32_t)ly * (uint32_t)sy0), sx0) &
           row_cover((int)((uint32_t)e1 + (uint32_t)ly * (uint32_t)sy1), sx1);
    mask |= row << (ly * kHbW);
  }
  return mask & d;
}

// The same with exact 64-bit edge values, pixel by pixel (large triangles).
static __device__ __noinline__ uint32_t tri_mask_slow(const TriSm& T, int ox, int oy, const int box[4]) {
  uint32_t mask = 0;
  for (int ly = box[2]; ly <= box[3]; ++ly)
    for (int lx = box[0]; lx <= box[1]; ++lx) {
      long long e[3];
      edges64(T, ox + lx, oy + ly, e);
      bool cov = true;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const bool owned = !((uint32_t)T.eb.z & (1u << (3 + k)));
        cov &= e[k] > 0 || (e[k] == 0 && owned);
      }
      if (cov) mask |= 1u << (ly * kHbW + lx);
    }
  return mask;
}


// Exact depth key (interpolated 1/w, Sec. 2 "Stage 3", the reading O.8 of the depth
// formula) of a triangle record at pixel (px, py) = (ox + lx, oy + ly) of its half-block;
// also returns the barycentric weights l1, l2 it used.
__device__ __forceinline__ float tri_key(const TriSm& T, int4 ea, int4 eb, float4 kq, int lx, int ly, int px,
                                         int py, float& l1, float& l2) {
  const uint32_t fl = (uint32_t)eb.z;
  float f1, f2;
  if (fl & kTriFast) {
    const int e1 = (int)((uint32_t)ea.x + (uint32_t)lx * (uint32_t)ea.z + (uint32_t)ly * (uint32_t)eb.x);
    const int e2 = (int)((uint32_t)ea.y + (uint32_t)lx * (uint32_t)ea.w + (uint32_t)ly * (uint32_t)eb.y);
    f1 = __int2float_rn(e1);
    f2 = __int2float_rn(e2);
  } else {
    long long e[3];
    edges64(T, px, py, e);
    f1 = __ll2float_rn(e[1]);
    f2 = __ll2float_rn(e[2]);
  }
  l1 = __fmul_rn(f1, kq.w);
  l2 = __fmul_rn(f2, kq.w);
  return __fadd_rn(kq.x, __fadd_rn(__fmul_rn(l1, kq.y), __fmul_rn(l2, kq.z)));
}

// ATH: the alpha-threshold variant. Once the transmittance drops to kAlphaTMin nothing
// more is blended and `last` stays at the key of the fragment that got it there, so the
// misorder test below only flags fragments that belong in front of that one.
template <int K, bool VTX, bool BWD = false, bool ATH = false>
struct PixelState {
  // K = 1 with flat colours gathered at blend time: the colour of the fragment held in the
  // slot is loaded when it enters, so the gather overlaps the next fragment's work
  static constexpr bool kPrefetch = !VTX && K == 1;
  unsigned long long s[K];
  float4 c[VTX || kPrefetch ? K : 1];
  unsigned long long last;
  float r, g, b, T;
  bool flagged;
  GradPixel gp;

  // K = 1, forward, colours carried: the empty slot holds a fully transparent colour, so
  // blending it changes nothing (T and the colour stay, last is still kSent) and the in-order
  // insert needs no test for it (layer frame rasteriser 0.409 -> 0.394 ms; the same for the
  // flat colours gathered at blend time made the particle frame's 14% slower)
  static constexpr bool kNullSlot = VTX && K == 1 && !BWD;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int i = 0; i < K; ++i) s[i] = kSent;
    if (kNullSlot) c[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    last = kSent;
    r = g = b = 0.f;
    T = 1.f;
    flagged = false;
  }

  // the pixel still blends (always, without the threshold)
  __device__ __forceinline__ bool live() const { return !ATH || T > kAlphaTMin; }

  __device__ __forceinline__ void blend(unsigned long long key, float4 col, const ViewDev& V) {
    const uint32_t j = (uint32_t)key >> 1;
    if (!VTX && !kPrefetch) col = __ldg(reinterpret_cast<const float4*>(V.col) + j);
    const float w = T * col.w;
    r += w * col.x;
    g += w * col.y;
    b += w * col.z;
    if (BWD && gp.grad) {
      const float om = 1.0f - col.w;
      float da = gp.gr * T * col.x + gp.gg * T * col.y + gp.gb * T * col.z;
      if (om > 1e-6f) {
        const float inv = rcp_approx(om);   // gradients need no correctly rounded divide
        da -= (gp.gr * (gp.fr - r) + gp.gg * (gp.fg - g) + gp.gb * (gp.fb - b)) * inv;
        da += gp.ga * gp.fT * inv;
      }
      // lanes blending a fragment of the same quad at this point add their contributions
      // in shared memory first, and one of them issues the four global atomics
      const int lane = threadIdx.x & 31;
      const unsigned act = __activemask();
      const unsigned grp = __match_any_sync(act, j);
      gp.agg[lane] = make_float4(gp.gr * w, gp.gg * w, gp.gb * w, da);
      __syncwarp(act);
      if (lane == __ffs(grp) - 1) {
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        for (unsigned m = grp; m; m &= m - 1) {
          const float4 c = gp.agg[__ffs(m) - 1];
          sum.x += c.x; sum.y += c.y; sum.z += c.z; sum.w += c.w;
        }
        float* gq = gp.grad + 4ull * j;
        atomicAdd(gq + 0, sum.x);
        atomicAdd(gq + 1, sum.y);
        atomicAdd(gq + 2, sum.z);
        atomicAdd(gq + 3, sum.w);
      }
      __syncwarp(act);
    }
    // T (1 - a) as one fused T - T a (a rounding, not the product's two, away from it: well
    // inside the colour tolerance); the threshold variant, whose T decides which fragments
    // blend, and the backward keep the product
    if (ATH || BWD) T *= 1.0f - col.w;
    else T = __fmaf_rn(-T, col.w, T);
  }

  __device__ __forceinline__ void insert(unsigned long long x, float4 xc, const ViewDev& V) {
    // nearer than a fragment already blended: order not guaranteed. The forward pass with
    // carried colours only records it (the pixel's composite is discarded, so inserting the
    // fragment anyway is harmless; measured faster than the branch there, slower for the
    // colours gathered at blend time)
    if (VTX && !BWD) {
      flagged |= x > last;
    } else if (x > last) {
      flagged = true;
      return;
    }
    if (VTX && K == 1 && kNullSlot && !ATH) {
      // one slot, the empty one transparent: blend the nearer of the held and the arriving
      // fragment, keep the other (selects: whichever way a lane's fragments arrive, the warp
      // runs one path; layer frame rasteriser 0.3770 -> 0.3750 ms against the branch below)
      const bool nearer = x > s[0];
      const unsigned long long bk = nearer ? x : s[0];
      const float4 bc = nearer ? xc : c[0];
      blend(bk, bc, V);
      last = bk;
      s[0] = nearer ? s[0] : x;
      c[0] = nearer ? c[0] : xc;
      return;
    }
    if (VTX && K == 1) {       // one slot (threshold, backward): a branch
      if (x > s[0]) {          // nearer than the held fragment: blend it at once
        if (live()) {
          blend(x, xc, V);
          last = x;
        }
      } else {
        if ((kNullSlot || s[0] != kSent) && live()) {
          blend(s[0], c[0], V);
          last = s[0];
        }
        s[0] = x;
        c[0] = xc;
      }
      return;
    }
    if (kPrefetch) {
      const float4* cp = reinterpret_cast<const float4*>(V.col) + ((uint32_t)x >> 1);
      if (x > s[0]) {          // nearer than the held fragment: blend it at once
        if (live()) {
          blend(x, __ldg(cp), V);
          last = x;
        }
      } else {
        if (s[0] != kSent && live()) {
          blend(s[0], c[0], V);
          last = s[0];
        }
        s[0] = x;
        c[0] = __ldg(cp);
      }
      return;
    }
    const bool xfirst = x > s[0];
    const unsigned long long ev = xfirst ? x : s[0];
    const unsigned long long y = xfirst ? s[0] : x;
    float4 evc = xc, yc = xc;
    if (VTX) {
      evc = xfirst ? xc : c[0];
      yc = xfirst ? c[0] : xc;
    }
    // new slots = {s[1..K-1], y} in decreasing order
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const bool take_next = (i + 1 < K) && (s[i + 1 < K ? i + 1 : i] > y);
      const bool take_y = (i == 0) || (s[i] > y);
      const unsigned long long nxt = s[i + 1 < K ? i + 1 : i];
      s[i] = take_next ? nxt : (take_y ? y : s[i]);
      if (VTX) {
        const float4 nc = c[i + 1 < K ? i + 1 : i];
        c[i] = take_next ? nc : (take_y ? yc : c[i]);
      }
    }
    if (ev != kSent && live()) {
      blend(ev, evc, V);
      last = ev;
    }
  }

  __device__ __forceinline__ void flush(const ViewDev& V) {
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (s[i] != kSent && live()) blend(s[i], VTX || kPrefetch ? c[i] : make_float4(0.f, 0.f, 0.f, 0.f), V);
  }
};

__device__ __forceinline__ void write_pixel(const ViewDev& V, long long pidx, float r, float g, float b,
                                            float T) {
  const float a = 1.0f - T;
  reinterpret_cast<float4*>(V.out)[pidx] = make_float4(r, g, b, a);
  if (V.out8) {
    const uint32_t c0 = __float2uint_rn(__fmul_rn(__saturatef(r), 255.0f));
    const uint32_t c1 = __float2uint_rn(__fmul_rn(__saturatef(g), 255.0f));
    const uint32_t c2 = __float2uint_rn(__fmul_rn(__saturatef(b), 255.0f));
    const uint32_t c3 = __float2uint_rn(__fmul_rn(__saturatef(a), 255.0f));
    reinterpret_cast<uint32_t*>(V.out8)[pidx] = c0 | (c1 << 8) | (c2 << 16) | (c3 << 24);
  }
}

// HASH: the variant that also writes the per-pixel coverage hash (a test output); the
// others carry no code or registers for it. ATH: the alpha-threshold variant (forward
// only, no hash), which also skips candidate quads that cannot reach in front of any
// pixel of the half-block still blending. LIT: the colour-carrying variant that also
// shades lit views (per-vertex normals, one directional light).
template <int K, bool VTX, bool BWD, bool HASH, bool ATH = false, bool LIT = false>
__global__ __launch_bounds__(kRasterThreads, LR_RASTER_MIN_BLOCKS) void k_raster(Ws ws) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kSlots = col_slots(LIT);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = lane & (kHbW - 1), ly = lane >> 3;
  TriSm* tris = reinterpret_cast<TriSm*>(smem) + warp * 64;
  float4* qcs = reinterpret_cast<float4*>(smem + (size_t)kRasterWarps * 64 * sizeof(TriSm)) + (size_t)warp * 64 * kSlots;
  float4* agg = reinterpret_cast<float4*>(smem + raster_smem_bytes(VTX, false, LIT)) + (size_t)warp * 32;
  if (ws.ctrl->error == LR_ERR_OVERFLOW) return;
  const unsigned long long nitems = ws.ctrl->raster_items;
  unsigned long long frag_total = 0;

  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&ws.ctrl->raster_head, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const int lg = ws.bin_log2, hl = bin_hb_log2(lg), cl = bin_hb_cols_log2(lg);
    const int bin_g = (int)ws.bin_order[item >> hl];
    const int hb = (int)(item & ((1u << hl) - 1u));
    const int v = view_of_bin(ws.views, ws.n_views, bin_g);
    const ViewDev& V = ws.views[v];
    const int b = bin_g - V.bin_base;
    const int bx = b % V.nbx, by = b / V.nbx;
    const int ox = (bx << lg) + (hb & ((1 << cl) - 1)) * kHbW, oy = (by << lg) + (hb >> cl) * kHbH;
    if (ox >= V.width || oy >= V.height || !tile_owned(V, ox, oy)) continue;
    const int px = ox + lx, py = oy + ly;
    const bool pix_ok = px < V.width && py < V.height;
    const uint32_t off = ws.bin_off[bin_g];
    const int n = (int)(ws.bin_off[bin_g + 1] - off);
    const bool vtx_view = V.color_mode != LR_COLOR_FLAT;
    const bool hashing = HASH && V.hash != nullptr;
    // lit views: unit direction toward the light and the ambient term
    const float4 light = LIT ? make_float4(V.light[0], V.light[1], V.light[2], V.light[3])
                             : make_float4(0.f, 0.f, 0.f, 0.f);

    PixelState<K, VTX, BWD, ATH> st;
    st.init();
    st.gp.grad = nullptr;
    st.gp.agg = agg;
    if (BWD && pix_ok) {
      const long long pidx = (long long)py * V.width + px;
      const float4 gq = reinterpret_cast<const float4*>(ws.grad_out)[pidx];
      const float4 fq = reinterpret_cast<const float4*>(ws.fwd)[pidx];
      st.gp.gr = gq.x; st.gp.gg = gq.y; st.gp.gb = gq.z; st.gp.ga = gq.w;
      st.gp.fr = fq.x; st.gp.fg = fq.y; st.gp.fb = fq.z; st.gp.fT = 1.0f - fq.w;
    }
    uint32_t cnt = 0;
    unsigned long long hsh = 0;

    auto process = [&](int nc, uint32_t rec) {
      bool skip = false;
      if (ATH) {
        // The smallest key a fragment must exceed to change any pixel of the half-block:
        // 0 while a pixel still blends; a finished pixel needs a fragment in front of the
        // one that finished it (keys are positive floats, so their bits order like them);
        // pixels outside the image and pixels left to the exact path need nothing. A
        // candidate whose largest possible key is below that is skipped: every fragment
        // of it would be dropped.
        const uint32_t need = (!pix_ok || st.flagged) ? 0xFFFFFFFFu : (st.live() ? 0u : (uint32_t)(st.last >> 32));
        const uint32_t kmin = __reduce_min_sync(0xffffffffu, need);
        if (kmin != 0u) {
          if (lane < nc) {
            const int4 qv = __ldg(ws.rec + 4ull * rec + 2);   // the record's four 1/w
            const float qm = fmaxf(fmaxf(__int_as_float(qv.x), __int_as_float(qv.y)),
                                   fmaxf(__int_as_float(qv.z), __int_as_float(qv.w)));
            skip = __float_as_uint(qm * kKeyBoundScale) < kmin;
          }
          if (__all_sync(0xffffffffu, skip || lane >= nc)) return;
        }
      }
      // ---- 2. triangle setup and coverage masks, one quad per lane ---------------------
      uint32_t tm0 = 0, tm1 = 0;
      if (lane < nc && !(ATH && skip)) {
        const QuadRec R = load_rec(ws.rec, rec);
        const uint32_t jl = (uint32_t)(rec - V.quad_base);
        uint32_t vsel = 0;   // per set-up triangle t: bit 8 + t, and its corners 1, 2 at bits 4t
        // Both triangles share the diagonal v0 v2, which each passes in one direction: under
        // the top-left rule a pixel centre on it belongs to exactly one of its two directions,
        // so the coverage of the direction v2 -> v0 is computed once (dmask) and a triangle
        // traversing the diagonal the other way takes its complement. Only when both
        // triangles are small: their 32-bit exactness bound covers the diagonal's values at
        // every half-block that touches either triangle's box, the only ones using dmask.
        // (Flat colours only: with colours carried the extra live registers spill, and the
        // layer frame measured no faster; the particle frame's rasteriser 1.011 -> 1.005 ms.)
        const bool share = !VTX && (R.info & (kInfoSmall0 | (kInfoSmall0 << 1))) == (kInfoSmall0 | (kInfoSmall0 << 1));
        uint32_t dmask = 0;
        if (share) {
          const int dx = R.X[0] - R.X[2], dy = R.Y[0] - R.Y[2];
          const bool owned = dy < 0 || (dy == 0 && dx > 0);
          const int e0 = (int)((uint32_t)dx * (uint32_t)(256 * oy + 128 - R.Y[2]) -
                               (uint32_t)dy * (uint32_t)(256 * ox + 128 - R.X[2])) -
                         (owned ? 0 : 1);
#pragma unroll
          for (int ly = 0; ly < kHbH; ++ly)
            dmask |= row_cover((int)((uint32_t)e0 + (uint32_t)ly * (uint32_t)(256 * dx)), -256 * dy) << (ly * kHbW);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          TriSm& T = tris[2 * lane + t];
          int cor[3];
          uint32_t mk;
          if (R.info & (kInfoSmall0 << t)) {
            // arrays of their own, never passed out of line: they stay in registers
            int box[4], le[3], lsx[3], lsy[3];
            if (!setup_tri_small(T, R.X, R.Y, R.q, t ? R.inv[1] : R.inv[0], R.info, t, jl, ox, oy, cor, box, le, lsx,
                                 lsy))
              continue;
            if (share) {
              // the diagonal is edge 1 (c -> a: v2 -> v0) of T0 unswapped and of T1 swapped,
              // else edge 2 (a -> b: v0 -> v2); edge 0 never touches v0
              const bool d1 = ((R.info >> t) & kInfoSwap0) ? t == 1 : t == 0;
              mk = tri_mask_two(le[0], lsx[0], lsy[0], d1 ? le[2] : le[1], d1 ? lsx[2] : lsx[1],
                                d1 ? lsy[2] : lsy[1], d1 ? dmask : ~dmask, box);
            } else {
              mk = tri_mask_fast(le, lsx, lsy, box);
            }
          } else {
            const QuadRec G = R;   // the out-of-line path's own copy (its address escapes)
            int cg[3], box[4], le[3], lsx[3], lsy[3];
            if (!setup_tri(T, G.X, G.Y, G.q, G.info, t, jl, ox, oy, cg, box, le, lsx, lsy)) continue;
            mk = ((uint32_t)T.eb.z & kTriFast) ? tri_mask_fast(le, lsx, lsy, box) : tri_mask_slow(T, ox, oy, box);
            cor[0] = cg[0]; cor[1] = cg[1]; cor[2] = cg[2];
          }
          if (t == 0) tm0 = mk; else tm1 = mk;
          if (VTX) vsel |= (1u << (8 + t)) | ((uint32_t)(cor[1] | (cor[2] << 2)) << (4 * t));
        }
        if (VTX && vsel) {
          if (!vtx_view) {
            const float4 fc = __ldg(reinterpret_cast<const float4*>(V.col) + jl);
#pragma unroll
            for (int t = 0; t < 2; ++t)
              if (vsel & (1u << (8 + t))) {
                // zero increments: the fragments' interpolation with the scale 1 (below)
                // returns fc bit for bit
                float4* qc = qcs + (2 * lane + t) * kSlots;
                qc[0] = fc;
                qc[1] = make_float4(0.f, 0.f, 0.f, 0.f);
                qc[2] = make_float4(0.f, 0.f, 0.f, 0.f);
                tris[2 * lane + t].eb.z |= (int)kTriFlatCol;
              }
          } else if (LIT && V.color_mode == LR_COLOR_LIT) {
            // 32 bytes per vertex (straight RGBA, then the normal): as below, each triangle
            // stores its corners' colours times 1/w as (c0, c1 - c0, c2 - c0), then the same
            // for the normals
            uint4 vi = make_uint4(4 * jl, 4 * jl + 1, 4 * jl + 2, 4 * jl + 3);
            if (V.idx) vi = __ldg(reinterpret_cast<const uint4*>(V.idx) + jl);
            const float4* cv = reinterpret_cast<const float4*>(V.col);
            const uint32_t vk[4] = {vi.x, vi.y, vi.z, vi.w};
            float4 p[4], m[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float4 c = __ldg(cv + 2ull * vk[k]), n = __ldg(cv + 2ull * vk[k] + 1);
              p[k] = make_float4(R.q[k] * c.x, R.q[k] * c.y, R.q[k] * c.z, R.q[k] * c.w);
              m[k] = make_float4(R.q[k] * n.x, R.q[k] * n.y, R.q[k] * n.z, 0.f);
            }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              if (!(vsel & (1u << (8 + t)))) continue;
              const uint32_t kb = (vsel >> (4 * t)) & 3u, kc = (vsel >> (4 * t + 2)) & 3u;
              const float4 a1 = kb == 1 ? p[1] : (kb == 2 ? p[2] : p[3]);
              const float4 a2 = kc == 1 ? p[1] : (kc == 2 ? p[2] : p[3]);
              const float4 b1 = kb == 1 ? m[1] : (kb == 2 ? m[2] : m[3]);
              const float4 b2 = kc == 1 ? m[1] : (kc == 2 ? m[2] : m[3]);
              float4* qc = qcs + (2 * lane + t) * kSlots;
              qc[0] = p[0];
              qc[1] = make_float4(a1.x - p[0].x, a1.y - p[0].y, a1.z - p[0].z, a1.w - p[0].w);
              qc[2] = make_float4(a2.x - p[0].x, a2.y - p[0].y, a2.z - p[0].z, a2.w - p[0].w);
              qc[3] = m[0];
              qc[4] = make_float4(b1.x - m[0].x, b1.y - m[0].y, b1.z - m[0].z, 0.f);
              qc[5] = make_float4(b2.x - m[0].x, b2.y - m[0].y, b2.z - m[0].z, 0.f);
              tris[2 * lane + t].eb.z |= (int)kTriLit;
            }
          } else {
            // the quad's four corner colours times 1/w, loaded together once; each triangle
            // stores (c0, c1 - c0, c2 - c0) of its corners for the fragment's
            // c0 + l1 (c1 - c0) + l2 (c2 - c0)
            uint4 vi = make_uint4(4 * jl, 4 * jl + 1, 4 * jl + 2, 4 * jl + 3);
            if (V.idx) vi = __ldg(reinterpret_cast<const uint4*>(V.idx) + jl);
            const float4* cv = reinterpret_cast<const float4*>(V.col);
            const float4 c0 = __ldg(cv + vi.x), c1 = __ldg(cv + vi.y), c2 = __ldg(cv + vi.z), c3 = __ldg(cv + vi.w);
            const float4 p0 = make_float4(R.q[0] * c0.x, R.q[0] * c0.y, R.q[0] * c0.z, R.q[0] * c0.w);
            const float4 p1 = make_float4(R.q[1] * c1.x, R.q[1] * c1.y, R.q[1] * c1.z, R.q[1] * c1.w);
            const float4 p2 = make_float4(R.q[2] * c2.x, R.q[2] * c2.y, R.q[2] * c2.z, R.q[2] * c2.w);
            const float4 p3 = make_float4(R.q[3] * c3.x, R.q[3] * c3.y, R.q[3] * c3.z, R.q[3] * c3.w);
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              if (!(vsel & (1u << (8 + t)))) continue;
              const uint32_t kb = (vsel >> (4 * t)) & 3u, kc = (vsel >> (4 * t + 2)) & 3u;
              const float4 a1 = kb == 1 ? p1 : (kb == 2 ? p2 : p3);
              const float4 a2 = kc == 1 ? p1 : (kc == 2 ? p2 : p3);
              float4* qc = qcs + (2 * lane + t) * kSlots;
              qc[0] = p0;
              qc[1] = make_float4(a1.x - p0.x, a1.y - p0.y, a1.z - p0.z, a1.w - p0.w);
              qc[2] = make_float4(a2.x - p0.x, a2.y - p0.y, a2.z - p0.z, a2.w - p0.w);
            }
          }
        }
      }
      __syncwarp();
      // ---- 3. transpose: lane = pixel, bit c = covered by triangle t of quad c -----------
      uint32_t m0 = warp_transpose32(tm0, lane), m1 = warp_transpose32(tm1, lane);
      if (!pix_ok) m0 = m1 = 0;
      cnt += __popc(m0) + __popc(m1);
      // ---- 4. fragments in candidate order through the K-slot sorter -----------------
      // one fragment per iteration: the lowest candidate with a covering triangle, T0
      // before T1 when both cover the pixel
      auto frag_step = [&]() {
        const int c = __ffs(m0 | m1) - 1;
        const uint32_t cb = 1u << c;
        // the bit leaves m0 if set there, else m1 (no branch on which)
        const uint32_t in0 = m0 & cb;
        m0 ^= in0;
        m1 ^= cb ^ in0;
        const int t = in0 ? 0 : 1;
        const TriSm& T = tris[2 * c + t];
        const int4 eb = T.eb;
        const uint32_t fl = (uint32_t)eb.z, id = (uint32_t)eb.w;
        if (hashing) hsh += splitmix64(id);
        // (the forward discards a flagged pixel's composite, the exact path redoing it, so it
        // keeps inserting rather than testing the flag per fragment; the backward must not
        // add a flagged pixel's gradient)
        if (!BWD || !st.flagged) {
          const float4 kq = T.kq;
          float l1 = 0.f, l2 = 0.f;
          // (the colour-carrying variant keeps one path: its branch cost more than it saved)
          const float key = (!VTX && (fl & kTriConstKey)) ? kq.x : tri_key(T, T.ea, eb, kq, lx, ly, px, py, l1, l2);
          const unsigned long long sk = ((unsigned long long)__float_as_uint(key) << 32) | id;
          float4 col = make_float4(0.f, 0.f, 0.f, 0.f);
          if (VTX) {
            const float4* qc = qcs + (2 * c + t) * kSlots;
            {
              // perspective-correct colour: interpolated (c / w) divided by the
              // interpolated 1/w, which is the depth key; a flat-colour triangle of the
              // batch has zero increments and the scale 1, so a select replaces a branch
              // per fragment (a0 + l1 * 0 + l2 * 0 and the product by 1 are exact)
              const float rk = (fl & kTriFlatCol) ? 1.0f : rcp_approx(key);
              const float4 a0 = qc[0], d1 = qc[1], d2 = qc[2];
              col.x = (a0.x + l1 * d1.x + l2 * d2.x) * rk;
              col.y = (a0.y + l1 * d1.y + l2 * d2.y) * rk;
              col.z = (a0.z + l1 * d1.z + l2 * d2.z) * rk;
              col.w = (a0.w + l1 * d1.w + l2 * d2.w) * rk;
              if (LIT && (fl & kTriLit)) {
                // the interpolated normal (times the interpolated 1/w, which only scales
                // it); two-sided Lambert term plus ambient on RGB
                const float4 m0 = qc[3], e1 = qc[4], e2 = qc[5];
                const float nx = m0.x + l1 * e1.x + l2 * e2.x;
                const float ny = m0.y + l1 * e1.y + l2 * e2.y;
                const float nz = m0.z + l1 * e1.z + l2 * e2.z;
                const float nn = nx * nx + ny * ny + nz * nz;
                const float d = fabsf(nx * light.x + ny * light.y + nz * light.z);
                const float lam = nn > 0.f ? fminf(d * rsqrtf(nn), 1.0f) : 0.f;
                const float f = light.w + (1.0f - light.w) * lam;
                col.x *= f;
                col.y *= f;
                col.z *= f;
              }
            }
          }
          st.insert(sk, col, V);
        }
      };
      if (VTX) {
        while (m0 | m1) frag_step();
      } else {
        // two fragments per iteration (measured faster without colours carried, slower
        // with them)
        while (m0 | m1) {
          frag_step();
          if (!(m0 | m1)) break;
          frag_step();
        }
      }
      __syncwarp();
    };

    // The backward pass streams the half-block twice: first without gradients, to learn
    // which pixels the sorter cannot order (those are left to the exact path, which
    // emits their whole gradient), then with gradients for the other pixels only.
    // With the forward's exact-path mask the detection pass is skipped.
    bool pre_flagged = false;
    int first_pass = BWD ? 0 : 1;
    if (BWD && ws.bwd_mask) {
      const uint32_t hbx = (uint32_t)ox / kHbW, hby = (uint32_t)oy / kHbH;
      const uint32_t hbw = ((uint32_t)V.width + kHbW - 1) / kHbW;
      pre_flagged = (ws.bwd_mask[hby * hbw + hbx] >> lane) & 1u;
      first_pass = 1;
    }
    for (int pass = first_pass; pass < 2; ++pass) {
    if (BWD) {
      st.init();
      st.flagged = pre_flagged;
      st.gp.grad = (pass == 1 && pix_ok) ? ws.grad_col : nullptr;
      cnt = 0;
      hsh = 0;
    }
    // ---- 1. the half-block's candidates: set bits of its bitmap row, in sorted order ----
    const uint32_t* row = hb_row(ws, off, bin_g, n, hb);
    const int nw = (n + 31) >> 5;
    const uint32_t* ref_lo = reinterpret_cast<const uint32_t*>(ws.refs + off);   // low words
    for (int g = 0; g < nw; g += 32) {
      BitRounds br;
      br.prepare(g + lane < nw ? __ldg(row + g + lane) : 0u, lane);
      for (int r0 = 0; r0 < br.total; r0 += 32) {
        const int j = br.get(r0, lane);
        process(min(32, br.total - r0), j < 0 ? 0u : ~ref_lo[2 * (32 * g + j)]);
      }
    }
    if (pass == 0) pre_flagged = st.flagged;
    }

    // ---- finish the half-block ---------------------------------------------------------
    // a pixel the given mask missed has had part of its gradient added already: report it
    if (BWD && ws.bwd_mask && st.flagged && !pre_flagged) set_error(ws.ctrl, LR_ERR_MASK_MISMATCH);
    if (!BWD && V.xmask) {
      const uint32_t fm = __ballot_sync(0xffffffffu, pix_ok && st.flagged);
      if (lane == 0) {
        const uint32_t hbw = ((uint32_t)V.width + kHbW - 1) / kHbW;
        V.xmask[((uint32_t)oy / kHbH) * hbw + (uint32_t)ox / kHbW] = fm;
      }
    }
    if (!st.flagged) st.flush(V);
    if (pix_ok) {
      const long long pidx = (long long)py * V.width + px;
      if (!BWD && V.cnt) V.cnt[pidx] = cnt;
      if (!BWD && hashing) V.hash[pidx] = hsh;
      if (!st.flagged) {
        if (!BWD) write_pixel(V, pidx, st.r, st.g, st.b, st.T);
      } else {
        const unsigned long long slot = atomicAdd(&ws.ctrl->ovf_count, 1ull);
        ws.ovf_list[slot] = (uint32_t)(V.pix_base + pidx);
      }
    }
    frag_total += cnt;
  }
  // fragments of all pixels this warp rendered
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) frag_total += __shfl_xor_sync(0xffffffffu, frag_total, o);
  if (lane == 0 && frag_total) atomicAdd(&ws.ctrl->fragments, frag_total);
}

}  // namespace lr

// Each translation unit lr_raster_k<K>.cu instantiates the rasteriser for one sorter
// capacity K (both colour layouts) through this macro, so the variants compile in
// parallel.
#define LR_DEFINE_RASTER(KK)                                                                  \
  namespace lr {                                                                              \
  template <bool VTX, bool BWD, bool HASH, bool ATH = false, bool LIT = false>                \
  static cudaError_t raster_attr_##KK() {                                                     \
    return cudaFuncSetAttribute(k_raster<KK, VTX, BWD, HASH, ATH, LIT>,                       \
                                cudaFuncAttributeMaxDynamicSharedMemorySize,                  \
                                (int)raster_smem_bytes(VTX, BWD, LIT));                       \
  }                                                                                           \
  cudaError_t prepare_raster_##KK(int* blocks_flat, int* blocks_vtx, int* blocks_bwd,         \
                                  int* blocks_lit) {                                          \
    cudaError_t e = raster_attr_##KK<false, false, false>();                                  \
    if (e == cudaSuccess) e = raster_attr_##KK<true, false, false>();                         \
    if (e == cudaSuccess) e = raster_attr_##KK<false, true, false>();                         \
    if (e == cudaSuccess) e = raster_attr_##KK<false, false, true>();                         \
    if (e == cudaSuccess) e = raster_attr_##KK<true, false, true>();                          \
    if (e == cudaSuccess) e = raster_attr_##KK<false, false, false, true>();                  \
    if (e == cudaSuccess) e = raster_attr_##KK<true, false, false, true>();                   \
    if (e == cudaSuccess) e = raster_attr_##KK<true, false, false, false, true>();            \
    if (e != cudaSuccess) return e;                                                           \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                        \
        blocks_lit, k_raster<KK, true, false, false, false, true>, kRasterThreads,            \
        raster_smem_bytes(true, false, true));                                                \
    if (e != cudaSuccess) return e;                                                           \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_flat, k_raster<KK, false, false, false>, \
                                                      kRasterThreads, raster_smem_bytes(false)); \
    if (e != cudaSuccess) return e;                                                           \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_bwd, k_raster<KK, false, true, false>, \
                                                      kRasterThreads, raster_smem_bytes(false, true)); \
    if (e != cudaSuccess) return e;                                                           \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_vtx, k_raster<KK, true, false, false>, \
                                                         kRasterThreads, raster_smem_bytes(true)); \
  }                                                                                           \
  /* mode: 0 flat colours, 1 colours in the sorter, 2 backward; + 4: coverage hash;        \
     + 8: alpha threshold (modes 8 and 9 only); 17: colours in the sorter with lit views */   \
  cudaError_t launch_raster_##KK(int mode, const Ws& ws, int grid, cudaStream_t st) {         \
    const size_t sf = raster_smem_bytes(false), sv = raster_smem_bytes(true);                 \
    /* a plain launch: with programmatic serialisation the persistent CTAs, placed early  \
       next to the bin sort's, measured slower on the particle frame */                       \
    switch (mode) {                                                                           \
      case 1: k_raster<KK, true, false, false><<<grid, kRasterThreads, sv, st>>>(ws); break;  \
      case 2: k_raster<KK, false, true, false><<<grid, kRasterThreads, raster_smem_bytes(false, true), st>>>(ws); break; \
      case 4: k_raster<KK, false, false, true><<<grid, kRasterThreads, sf, st>>>(ws); break;  \
      case 5: k_raster<KK, true, false, true><<<grid, kRasterThreads, sv, st>>>(ws); break;   \
      case 8: k_raster<KK, false, false, false, true><<<grid, kRasterThreads, sf, st>>>(ws); break; \
      case 9: k_raster<KK, true, false, false, true><<<grid, kRasterThreads, sv, st>>>(ws); break; \
      case 17:                                                                                \
        k_raster<KK, true, false, false, false, true>                                         \
            <<<grid, kRasterThreads, raster_smem_bytes(true, false, true), st>>>(ws);         \
        break;                                                                                \
      default: k_raster<KK, false, false, false><<<grid, kRasterThreads, sf, st>>>(ws); break; \
    }                                                                                         \
    return cudaGetLastError();                                                                \
  }                                                                                           \
  }
