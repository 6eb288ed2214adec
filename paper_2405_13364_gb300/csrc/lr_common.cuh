// lr_common.cuh -- device-side data layout shared by the pipeline kernels.
//
// One render processes a batch of views (a single frame is a batch of one). Every stage
// runs as one launch over all views: quads, bins and pixels of all views live in
// flattened index spaces, and each view's slice starts at a base offset stored in its
// ViewDev record.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lr.h"

#include <utility>

namespace lr {

constexpr int kBinLog2Default = 5;          // 32x32-pixel bins (Sec. 2, Stage 2); 16 and 64
                                            // are the alternatives (lr_config.bin_size)
constexpr int kHbW = 8, kHbH = 4;           // 8x4 half-blocks (Sec. 2, Stage 3)
constexpr int kTileLog2 = 5;                // 32x32-pixel tiles of lr_view.owned_tiles

// Geometry of a bin of 2^lg pixels per side (lg = 4, 5 or 6): its 8x4 half-blocks, cols
// per row and rows, numbered hy * cols + hx; the transposed half-block bitmap of a bin
// keeps mrows >= 32 rows (a multiple of 32, so that a reference's half-block mask is mw
// whole 32-bit words).
__host__ __device__ __forceinline__ int bin_hb_log2(int lg) { return 2 * lg - 5; }            // 3, 5, 7
__host__ __device__ __forceinline__ int bin_hb(int lg) { return 1 << bin_hb_log2(lg); }       // 8, 32, 128
__host__ __device__ __forceinline__ int bin_hb_cols_log2(int lg) { return lg - 3; }           // 1, 2, 3
__host__ __device__ __forceinline__ int bin_hb_cols(int lg) { return 1 << (lg - 3); }         // 2, 4, 8
__host__ __device__ __forceinline__ int bin_mrows_log2(int lg) { return lg < 5 ? 5 : 2 * lg - 5; }
__host__ __device__ __forceinline__ int bin_mrows(int lg) { return 1 << bin_mrows_log2(lg); }  // 32, 32, 128
__host__ __device__ __forceinline__ int bin_mw(int lg) { return bin_mrows(lg) >> 5; }         // 1, 1, 4
constexpr float kGuardPx = 16384.0f;        // guard band, pixels
constexpr int kSortSmemCap = 2048;          // bins below this many refs: k_bin_sort (256 threads)
constexpr int kSortBigCap = 8192;           // k_bin_sort_big sorts runs of up to this many refs
constexpr int kSortBigThreads = 1024;
// k_bin_sort_big's bucket sort: at most this many buckets per bin, the largest bin sorted
// this way in shared memory, and the largest bucket sorted by insertion (a bin with a
// larger bucket, e.g. many equal depths, falls back to the merge sort)
constexpr int kBucketsBig = 4096;
constexpr int kBucketBigCap = 20480;
constexpr int kMaxBucket = 64;
constexpr size_t kSortSmemBytes = 2 * (size_t)kSortSmemCap * 8;
constexpr size_t kSortBigSmemBytes =
    (size_t)kBucketBigCap * 8 + (2 * (size_t)kBucketsBig + 2) * 4 > 2 * (size_t)kSortBigCap * 8
        ? (size_t)kBucketBigCap * 8 + (2 * (size_t)kBucketsBig + 2) * 4
        : 2 * (size_t)kSortBigCap * 8;
constexpr int kHistSmemBins = 8192;         // shared-memory bin counters per CTA (Sec. 2 Stage 2)
#ifndef LR_CHUNK_QUADS
#define LR_CHUNK_QUADS 2048
#endif
constexpr int kChunkQuads = LR_CHUNK_QUADS;  // quads per binning CTA
constexpr int kBinThreads = kChunkQuads / 4 < 1024 ? kChunkQuads / 4 : 1024;   // threads per binning CTA
constexpr int kBinMinBlocks = kBinThreads >= 1024 ? 1 : (kBinThreads >= 512 ? 2 : 5);
constexpr int kSmallBins = 4;               // AABB-counted up to kSmallBins x kSmallBins bins

// cull reasons (stats and rec_info bits 8..11)
enum Cull : uint32_t {
  kVisible = 0, kBadIndex = 1, kNonFinite = 2, kDepth = 3, kGuard = 4, kDegenerate = 5,
  kNoPixel = 6
};

// rec_info bits
constexpr uint32_t kInfoTri0 = 1u;          // triangle 0 has non-zero area
constexpr uint32_t kInfoTri1 = 2u;          // triangle 1 has non-zero area
constexpr uint32_t kInfoLarge = 4u;         // bin rectangle larger than kSmallBins^2 bins
constexpr uint32_t kInfoFlatDepth = 8u;     // all four vertices have the same 1/w
constexpr uint32_t kInfoSwap0 = 16u;        // triangle t (bit << t): negative area, v1 <-> v2
constexpr uint32_t kInfoSmall0 = 64u;       // triangle t (bit << t): 32-bit edge values are
                                            // exact on every half-block its box touches
constexpr uint32_t kRectInvisible = 0x0000FFFFu;   // rect.x value of a culled quad

struct ViewDev {
  const float* pos;          // f32[V][3]
  const uint32_t* idx;       // u32[Q][4] or nullptr
  const float* col;          // flat f32[Q][4] or vertex f32[V][4]
  float* out;                // f32[H][W][4]
  uint8_t* out8;             // optional
  uint32_t* cnt;             // optional
  unsigned long long* hash;  // optional
  uint32_t* xmask;           // optional: exact-path bits per 8x4 half-block
  const uint32_t* owned;     // optional: bit set of the 32x32-pixel tiles to rasterise
  float m[12];               // rows 0, 1, 3 of the view-projection (x, y, w)
  float near_z, far_z;
  float half_w, half_h;
  long long num_vertices;
  long long quad_base;       // first record of this view in the flattened quad space
  long long pix_base;        // first pixel of this view in the flattened pixel space
  int num_quads;
  int color_mode;
  int width, height;
  int nbx, nby;              // bins per row / column
  int bin_base;              // first bin of this view in the flattened bin space
  int chunk_base;            // first binning chunk (kChunkQuads quads) of this view
  int sub_x, sub_y;          // multisampling: the view's sample offset from the pixel centre
                             // (1/256 px), subtracted from the snapped vertices, so that the
                             // pixel-centre tests of every later stage test the sample
  float light[4];            // lit colours: unit direction toward the light, ambient term
};

// Whether the 32x32-pixel tile holding pixel (px, py) is to be rasterised (every tile when
// the view has no owned-tile set).
__device__ __forceinline__ bool tile_owned(const ViewDev& V, int px, int py) {
  if (!V.owned) return true;
  const int t = (py >> kTileLog2) * ((V.width + 31) >> kTileLog2) + (px >> kTileLog2);
  return (__ldg(V.owned + (t >> 5)) >> (t & 31)) & 1u;
}

// Up to kViewsPerLaunch view descriptors passed by value to a kernel, which writes them to
// the workspace (no host buffer is needed).
constexpr int kViewsPerLaunch = 16;
struct ViewChunk {
  ViewDev v[kViewsPerLaunch];
  int first, count;
};

// Programmatic dependent launch (sm_90 and later). The pipeline's kernels (all but the
// rasteriser) are launched with programmatic stream serialisation (launch_pdl), so each
// may be scheduled while its predecessor in the stream drains; every kernel first waits
// for its predecessor's completion and memory (griddepcontrol.wait: nothing of the kernel
// touches memory before it), then lets its own successor begin launching. A kernel
// launched without the attribute passes both instructions at once. Contexts that render
// on several streams at once turn it off (LR_FLAG_NO_PDL): early-placed waiting CTAs would
// hold resources the other streams' kernels need.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                     cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Device control block at the start of the workspace.
struct Ctrl {
  int error;                         // first error (lr_status), 0 = none
  int pad0;
  unsigned long long refs_total;     // sum of bin counts = references needed
  unsigned long long refs_cap;
  unsigned long long raster_head;    // rasteriser work queue
  unsigned long long raster_items;
  unsigned long long ovf_count;      // pixels registered for the exact path
  unsigned long long ovf_head;
  unsigned long long sort_head;      // k_bin_sort_big's queue over the high-density bins
  unsigned long long fragments;
  unsigned long long unused0;
  unsigned long long culled[8];
  unsigned long long bins_nonempty;
  unsigned long long bins_high;
  unsigned long long max_bin;
  unsigned long long chunk_list_head;   // allocation cursor of the chunks' (bin, base) lists
  // high-density bins by the sort k_bin_sort_big gave them: bucket sort, merge sort in
  // shared memory alone, merge sort with runs merged through global memory
  unsigned long long sort_branch[3];
  unsigned long long pad[4];
};

// The per-quad record written by k_setup and gathered by every later stage, 64 bytes so
// that one quad is four 16-byte loads from one cache line:
//   w0 = (X0, Y0, X1, Y1), w1 = (X2, Y2, X3, Y3)  snapped vertices, 1/256 pixel
//   w2 = 1/w of vertices 0..3 (float bits)
//   w3 = (1 / (float)|A0|, 1 / (float)|A1| (float bits, 0 for a zero-area triangle), info, 0)
struct QuadRec {
  int X[4], Y[4];
  float q[4];
  float inv[2];
  uint32_t info;
};

__device__ __forceinline__ QuadRec load_rec(const int4* rec, uint32_t i) {
  const int4* p = rec + 4ull * i;
  const int4 a = p[0], b = p[1], c = p[2], d = p[3];
  QuadRec r;
  r.X[0] = a.x; r.Y[0] = a.y; r.X[1] = a.z; r.Y[1] = a.w;
  r.X[2] = b.x; r.Y[2] = b.y; r.X[3] = b.z; r.Y[3] = b.w;
  r.q[0] = __int_as_float(c.x); r.q[1] = __int_as_float(c.y);
  r.q[2] = __int_as_float(c.z); r.q[3] = __int_as_float(c.w);
  r.inv[0] = __int_as_float(d.x); r.inv[1] = __int_as_float(d.y);
  r.info = (uint32_t)d.z;
  return r;
}

// Pointers into the workspace for one render (passed by value to every kernel).
struct Ws {
  Ctrl* ctrl;
  const ViewDev* views;
  int n_views;
  int total_bins;
  long long total_quads;
  long long total_pix;
  long long refs_cap;
  int bin_log2;              // bins of 2^bin_log2 x 2^bin_log2 pixels (the same for every view)
  int4* rec;                 // [4 * total_quads]: the 64-byte quad record (QuadRec)
  uint2* rec_rect;           // [total_quads]: pixel AABB (px0 | px1 << 16, py0 | py1 << 16)
  uint32_t* rec_info;        // [total_quads]: kInfo* bits | cull reason << 8
  float* rec_rep;            // [total_quads]: representative 1/w over the quad's whole box
  uint32_t* bin_count;       // [total_bins]
  uint32_t* bin_off;         // [total_bins + 1]
  uint32_t* bin_cursor;      // [total_bins]
  uint2* chunk_span;         // [total_chunks] (start, length) of the chunk's list of (bin, base
                             // of the chunk's range within the bin), kept in refs_tmp
  uint32_t* bin_order;       // [total_bins]: bins by decreasing reference count
  unsigned long long* refs;      // [refs_cap] sorted per bin: (~rep_bits << 32) | ~record
  unsigned long long* refs_tmp;  // [refs_cap] merge buffer of the high-density sort
  uint32_t* ref_hb;          // [mw * refs_cap + mrows * total_bins] per bin, the transposed
                             // half-block bitmap of its sorted references (hb_row)
  uint32_t* ovf_list;        // [total_pix] flattened pixel ids registered for the exact path
  // backward
  const float* grad_out;     // f32[H][W][4] of view 0
  const float* fwd;          // f32[H][W][4] of view 0
  float* grad_col;           // f32[Q][4] of view 0
  const uint32_t* bwd_mask;  // optional: the forward's exact-path mask of view 0
  // alpha threshold: blend a fragment only while the pixel's transmittance is above t_min
  // (0: off, every fragment blended)
  float t_min;
};

// 32x32 bit-matrix transpose across a warp: lane r holds row r on entry (bit c = element
// (r, c)) and column r on exit (bit c = element (c, r)); five butterfly exchanges.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  const uint32_t m[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int j = 16 >> i;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~m[i]) | ((y >> j) & m[i])) : ((x & m[i]) | ((y & m[i]) << j));
  }
  return x;
}

// The half-block bitmap of a bin with n sorted references starting at off: row h (one per
// 8x4 half-block; bin_mrows rows) holds nw = ceil(n / 32) words, bit j of word w set iff
// reference 32 w + j overlaps half-block h. Rows of bin b start at mw * off + mrows * b, so
// the bitmaps of all bins fit in mw * refs + mrows * bins words.
__device__ __forceinline__ const uint32_t* hb_row(const Ws& ws, uint32_t off, int bin, int n, int hb) {
  const int ml = bin_mrows_log2(ws.bin_log2);
  return ws.ref_hb + ((size_t)off << (ml - 5)) + ((size_t)bin << ml) + (size_t)hb * (size_t)((n + 31) >> 5);
}

// Position of the k-th (0-based) set bit of m; k < popc(m).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int k) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    const int lc = __popc(m & ((1u << w) - 1u));
    if (k >= lc) {
      k -= lc;
      m >>= w;
      pos += w;
    }
  }
  return pos;
}

// Hands out the set bits of up to 32 bitmap words (one per lane, `word`) in order, 32 at a
// time: after prepare(), round r gives lane L the (32 r + L)-th set bit overall as a bit
// index 32 * (word's lane) + position, or -1 past the end.
struct BitRounds {
  uint32_t word;
  int incl;     // inclusive prefix of the set-bit counts over lanes
  int total;
  __device__ __forceinline__ void prepare(uint32_t w, int lane) {
    word = w;
    incl = __popc(w);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
  }
  __device__ __forceinline__ int get(int r0, int lane) const {
    const int p = r0 + lane;
    int s = 0;   // number of lanes whose inclusive count is <= p = the lane holding bit p
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int v = __shfl_sync(0xffffffffu, incl, s + step - 1);
      if (v <= p) s += step;
    }
    s = min(s, 31);
    const uint32_t ws = __shfl_sync(0xffffffffu, word, s);
    const int before = __shfl_sync(0xffffffffu, incl, s) - __popc(ws);
    if (p >= total) return -1;
    return 32 * s + nth_set_bit(ws, p - before);
  }
};

__device__ __forceinline__ void set_error(Ctrl* c, int code) { atomicCAS(&c->error, 0, code); }

// View owning a flattened quad / bin / pixel index (views are few; binary search).
__device__ __forceinline__ int view_of_quad(const ViewDev* v, int n, long long q) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (v[mid].quad_base <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int view_of_bin(const ViewDev* v, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (v[mid].bin_base <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int view_of_chunk(const ViewDev* v, int n, int c) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (v[mid].chunk_base <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int view_of_pixel(const ViewDev* v, int n, long long p) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (v[mid].pix_base <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// floor(a / 256) and ceil(a / 256) for signed 64-bit a
__device__ __forceinline__ int floor_div256(long long a) { return (int)(a >> 8); }
__device__ __forceinline__ int ceil_div256(long long a) { return (int)(-((-a) >> 8)); }

__device__ __forceinline__ long long area2(int xa, int ya, int xb, int yb, int xc, int yc) {
  return (long long)(xb - xa) * (long long)(yc - ya) - (long long)(yb - ya) * (long long)(xc - xa);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  // splitmix64 output function (Steele, Lea, Flood 2014; constants as published by Vigna)
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Approximate reciprocal (PTX rcp.approx.ftz.f32, about 1 ulp): colours, gradients and
// sort hints only, never coverage or the depth key.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Representative depth of a quad over a pixel box: the plane of one triangle evaluated (in
// plain fp32, approximately) at the box centre, clamped to the range of the quad's vertex
// 1/w. Only the order quality of stage 1 (the per-bin depth sort) depends on it; exactness
// is restored by the per-pixel sorter and the overflow path. The triangle's vertices are
// picked with selects, so the arrays stay in registers.
__device__ __forceinline__ float rep_depth_of(const int X[4], const int Y[4], const float Q[4], uint32_t info,
                                              int x0, int x1, int y0, int y1) {
  const bool t0 = (info & kInfoTri0) != 0;   // triangle (v0 v1 v2), else (v0 v2 v3)
  const float xa = (float)X[0], ya = (float)Y[0], qa = Q[0];
  const float xb = (float)(t0 ? X[1] : X[2]), yb = (float)(t0 ? Y[1] : Y[2]), qb = t0 ? Q[1] : Q[2];
  const float xc = (float)(t0 ? X[2] : X[3]), yc = (float)(t0 ? Y[2] : Y[3]), qc = t0 ? Q[2] : Q[3];
  const float qmin = fminf(fminf(Q[0], Q[1]), fminf(Q[2], Q[3]));
  const float qmax = fmaxf(fmaxf(Q[0], Q[1]), fmaxf(Q[2], Q[3]));
  const float px = 128.0f * (float)(x0 + x1) + 128.0f, py = 128.0f * (float)(y0 + y1) + 128.0f;
  const float A = (xb - xa) * (yc - ya) - (yb - ya) * (xc - xa);
  if (!(fabsf(A) > 0.0f)) return qmax;
  const float iA = rcp_approx(A);
  const float l1 = ((xa - xc) * (py - yc) - (ya - yc) * (px - xc)) * iA;
  const float l2 = ((xb - xa) * (py - ya) - (yb - ya) * (px - xa)) * iA;
  float r = qa + l1 * (qb - qa) + l2 * (qc - qa);
  r = fminf(fmaxf(r, qmin), qmax);
  return r > 0.0f ? r : qmin;
}

// Correctly rounded quotient a / w given y = 1/w rounded to nearest, by Markstein's
// correction (P. Markstein, "Computation of elementary functions on the IBM RISC System/6000
// processor", IBM J. Res. Dev. 34(1), 1990): if y is the correctly rounded reciprocal and q
// is within one ulp of a/w, then q + r y with the residual r = a - w q (exact in one fused
// multiply-add) rounds once to the correctly rounded quotient. q = a y can be two ulps off,
// so a first correction brings it within one ulp and a second one rounds it correctly. The
// theorem needs every operand, residual and the quotient to be normal numbers; anything
// outside the range tested below takes the IEEE division.
__device__ __forceinline__ float div_rn_by(float a, float w, float y) {
  const float q0 = __fmul_rn(a, y);
  const float aa = fabsf(a);
  if (!(w >= 0x1p-60f && w <= 0x1p60f && aa >= 0x1p-90f && aa <= 0x1p60f && fabsf(q0) >= 0x1p-60f))
    return __fdiv_rn(a, w);
  const float q1 = __fmaf_rn(__fmaf_rn(-q0, w, a), y, q0);
  return __fmaf_rn(__fmaf_rn(-q1, w, a), y, q1);
}

}  // namespace lr
