// lr_bin.cu -- Stage 2 of the pipeline, quad binning (Sec. 2, "Stage 2: quad binning"),
// plus the per-bin depth sort that feeds Stage 3.
//
//   k_bin_count    Phase 1: per-bin reference counts. Each CTA owns a chunk of 2048 quads
//                  of one view and counts into shared-memory bin counters (the paper's
//                  5120-entry arrays), then adds its non-zero counters to global memory.
//                  Quads whose bin rectangle is at most 4x4 bins are counted from their
//                  AABB; larger quads are tested bin by bin with a conservative
//                  per-triangle edge test (trivial reject), the whole warp sharing one
//                  large quad's bins.
//   k_bin_scan     Phase 2: exclusive scan of the counts into list offsets, capacity
//                  check, and a categorisation of bins by size (the paper's empty / low /
//                  high) that orders the rasteriser's work queue, largest bins first.
//   k_bin_scatter  Phase 3: places the chunk's references, each (chunk, bin) in the range
//                  k_bin_count reserved for it (k_bin_count's global atomic returns the
//                  range's base, listed per chunk), slots by shared-memory atomics. A
//                  reference is a 64-bit sort key:
//                  (~representative 1/w) << 32 | ~record index.
//   k_bin_sort     Stage-1 depth sort: sorts each bin's references ascending, i.e. front
//                  to back by a representative depth, ties with the higher quad index
//                  first. Bins with fewer than 2048 references: one 256-thread CTA per
//                  bin, a merge sort in shared memory (runs of 64 to 256 keys sorted in
//                  registers by one warp each, then merge-path levels).
//   k_bin_sort_big The high-density bins (2048 references or more; the paper's "high"
//                  category): persistent 1024-thread CTAs take them from the front of the
//                  size-ordered bin list. Up to 20480 references are bucket-sorted in
//                  shared memory (about two references per bucket between the bin's depth
//                  extremes, insertion sort per bucket); bins with a bucket over 64
//                  references (many equal depths) or longer lists merge-sort runs of up to
//                  8192 references in shared memory and merge them through a global buffer.
#include "lr_common.cuh"

namespace lr {

// Conservative test whether a triangle of a quad can cover a pixel centre of bin (bx, by):
// false only if one edge is negative (after the fill-rule bias) at all four corner pixel
// centres of the bin rectangle clipped to the triangle's pixel AABB and the screen.
__device__ bool tri_may_touch_bin(const int X[4], const int Y[4], int t, int bx, int by, int W, int H, int lg) {
  int a = 0, b = t == 0 ? 1 : 2, c = t == 0 ? 2 : 3;
  long long A = area2(X[a], Y[a], X[b], Y[b], X[c], Y[c]);
  if (A == 0) return false;
  if (A < 0) { int tmp = b; b = c; c = tmp; }
  const int vx[3] = {X[a], X[b], X[c]}, vy[3] = {Y[a], Y[b], Y[c]};
  const int xmin = min(vx[0], min(vx[1], vx[2])), xmax = max(vx[0], max(vx[1], vx[2]));
  const int ymin = min(vy[0], min(vy[1], vy[2])), ymax = max(vy[0], max(vy[1], vy[2]));
  const int x0 = max(max(ceil_div256((long long)xmin - 128), 0), bx << lg);
  const int x1 = min(min(floor_div256((long long)xmax - 128), W - 1), ((bx + 1) << lg) - 1);
  const int y0 = max(max(ceil_div256((long long)ymin - 128), 0), by << lg);
  const int y1 = min(min(floor_div256((long long)ymax - 128), H - 1), ((by + 1) << lg) - 1);
  if (x0 > x1 || y0 > y1) return false;
  const long long cx[2] = {256LL * x0 + 128, 256LL * x1 + 128};
  const long long cy[2] = {256LL * y0 + 128, 256LL * y1 + 128};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int u = e == 0 ? 1 : (e == 1 ? 2 : 0);
    const int w = e == 0 ? 2 : (e == 1 ? 0 : 1);
    const long long dx = (long long)vx[w] - vx[u], dy = (long long)vy[w] - vy[u];
    const long long bias = (dy < 0 || (dy == 0 && dx > 0)) ? 0 : -1;
    bool all_out = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long ev = dx * (cy[i >> 1] - vy[u]) - dy * (cx[i & 1] - vx[u]) + bias;
      all_out &= ev < 0;
    }
    if (all_out) return false;
  }
  return true;
}

__device__ __forceinline__ bool quad_may_touch_bin(const Ws& ws, long long q, uint32_t info, int bx,
                                                   int by, int W, int H) {
  const int4 a = ws.rec[4 * q], b = ws.rec[4 * q + 1];
  const int X[4] = {a.x, a.z, b.x, b.z}, Y[4] = {a.y, a.w, b.y, b.w};
  return ((info & kInfoTri0) && tri_may_touch_bin(X, Y, 0, bx, by, W, H, ws.bin_log2)) ||
         ((info & kInfoTri1) && tri_may_touch_bin(X, Y, 1, bx, by, W, H, ws.bin_log2));
}

// Per-bin representative depth of a quad that spans several bins.
__device__ __forceinline__ float rep_depth(const Ws& ws, long long q, uint32_t info, int x0, int x1,
                                           int y0, int y1) {
  const int4 a = ws.rec[4 * q], b = ws.rec[4 * q + 1], c = ws.rec[4 * q + 2];
  const int X[4] = {a.x, a.z, b.x, b.z}, Y[4] = {a.y, a.w, b.y, b.w};
  const float Q[4] = {__int_as_float(c.x), __int_as_float(c.y), __int_as_float(c.z), __int_as_float(c.w)};
  return rep_depth_of(X, Y, Q, info, x0, x1, y0, y1);
}

__device__ __forceinline__ unsigned long long ref_key(float rep, long long q) {
  return ((unsigned long long)(~__float_as_uint(rep)) << 32) | (unsigned long long)(~(uint32_t)q);
}

// Shared by count and scatter: for each (visible quad, touched bin) of the CTA's chunk
// call f(q, local_bin, bx, by). Small quads enumerate their AABB bins in their own
// thread; large quads are processed by the whole warp, one bin per lane.
// PF: the next iteration's rectangle and info are loaded while this one's bins are handled
// (the count's loop is latency-bound, a dependent load per iteration otherwise: 18.4 -> 17.0
// µs on the layer frame; the scatter, with more live registers, measured no faster with it).
template <bool PF, typename F>
__device__ __forceinline__ void for_each_ref(const Ws& ws, const ViewDev& V, long long q0, long long q1,
                                             F&& f) {
  const int lane = threadIdx.x & 31;
  const int lg = ws.bin_log2;
  long long base = q0 + (threadIdx.x & ~31);
  uint2 rect_n = make_uint2(kRectInvisible, kRectInvisible);
  uint32_t info_n = 0;
  if (PF && base + lane < q1) { rect_n = ws.rec_rect[base + lane]; info_n = ws.rec_info[base + lane]; }
  for (; base < q1; base += blockDim.x) {
    const long long q = base + lane;
    const bool in = q < q1;
    uint2 rect = rect_n;
    uint32_t info = info_n;
    if (PF) {
      rect_n = make_uint2(kRectInvisible, kRectInvisible);
      info_n = 0;
      if (q + blockDim.x < q1) { rect_n = ws.rec_rect[q + blockDim.x]; info_n = ws.rec_info[q + blockDim.x]; }
    } else if (in) {
      rect = ws.rec_rect[q];
      info = ws.rec_info[q];
    }
    const bool vis = in && rect.x != kRectInvisible;
    const int px0 = rect.x & 0xffff, px1 = rect.x >> 16, py0 = rect.y & 0xffff, py1 = rect.y >> 16;
    if (vis && !(info & kInfoLarge)) {
      for (int by = py0 >> lg; by <= (py1 >> lg); ++by)
        for (int bx = px0 >> lg; bx <= (px1 >> lg); ++bx) f(q, by * V.nbx + bx, bx, by, rect, info);
    }
    unsigned large = __ballot_sync(0xffffffffu, vis && (info & kInfoLarge));
    while (large) {
      const int src = __ffs(large) - 1;
      large &= large - 1;
      const long long lq = __shfl_sync(0xffffffffu, q, src);
      const uint2 lr = make_uint2(__shfl_sync(0xffffffffu, rect.x, src), __shfl_sync(0xffffffffu, rect.y, src));
      const uint32_t li = __shfl_sync(0xffffffffu, info, src);
      const int bx0 = (lr.x & 0xffff) >> lg, bx1 = (lr.x >> 16) >> lg;
      const int by0 = (lr.y & 0xffff) >> lg, by1 = (lr.y >> 16) >> lg;
      const int bw = bx1 - bx0 + 1, nb = bw * (by1 - by0 + 1);
      for (int i = lane; i < nb; i += 32) {
        const int bx = bx0 + i % bw, by = by0 + i / bw;
        if (quad_may_touch_bin(ws, lq, li, bx, by, V.width, V.height)) f(lq, by * V.nbx + bx, bx, by, lr, li);
      }
    }
  }
}

// count and scatter are latency-bound (gathers, atomics): chunks of 2048 quads on 512-thread
// CTAs, two per SM (measured a little faster than 1024 quads on 256 threads or 4096 on 1024)
__global__ __launch_bounds__(kBinThreads, kBinMinBlocks) void k_bin_count(Ws ws) {
  pdl_begin();
  __shared__ uint32_t hist[kHistSmemBins];
  const int v = view_of_chunk(ws.views, ws.n_views, blockIdx.x);
  const ViewDev& V = ws.views[v];
  const long long q0 = V.quad_base + (long long)(blockIdx.x - V.chunk_base) * kChunkQuads;
  const long long q1 = min(q0 + kChunkQuads, V.quad_base + V.num_quads);
  const int nb = V.nbx * V.nby;
  const bool smem = nb <= kHistSmemBins;
  if (smem)
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  for_each_ref<true>(ws, V, q0, q1, [&](long long, int b, int, int, uint2, uint32_t) {
    if (smem) atomicAdd(&hist[b], 1u);
    else atomicAdd(&ws.bin_count[V.bin_base + b], 1u);
  });
  __syncthreads();
  if (!smem) return;
  // reserve the chunk's range in every bin it touches, and list (bin, base of the range)
  // for k_bin_scatter, which then places references without recounting
  __shared__ uint32_t s_n, s_start, s_pos;
  if (threadIdx.x == 0) { s_n = 0; s_pos = 0; }
  __syncthreads();
  uint32_t mine = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) mine += hist[b] != 0u;
  if (mine) atomicAdd(&s_n, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    s_start = (uint32_t)min(atomicAdd(&ws.ctrl->chunk_list_head, (unsigned long long)s_n), 0xFFFFFFFFull);
    ws.chunk_span[blockIdx.x] = make_uint2(s_start, s_n);
  }
  __syncthreads();
  uint2* list = reinterpret_cast<uint2*>(ws.refs_tmp);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const uint32_t c = hist[b];
    if (!c) continue;
    const uint32_t base = atomicAdd(&ws.bin_count[V.bin_base + b], c);
    const unsigned long long at = (unsigned long long)s_start + atomicAdd(&s_pos, 1u);
    // a list past the reference capacity means the references do not fit either: the scan
    // reports the overflow and the scatter does not run
    if (at < (unsigned long long)ws.refs_cap) list[at] = make_uint2((uint32_t)b, base);
  }
}

// Single CTA. Offsets (exclusive scan), capacity check, and the bin order for the
// rasteriser: bins by decreasing size class (floor(log2(count)) + 1), empty bins last.
__global__ __launch_bounds__(1024) void k_bin_scan(Ws ws) {
  pdl_begin();
  __shared__ unsigned long long warp_sums[32];
  __shared__ uint32_t cls_count[34];
  __shared__ uint32_t cls_base[34];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = ws.total_bins;
  if (tid < 34) cls_count[tid] = 0;
  if (tid == 0) carry = 0;
  __syncthreads();
  unsigned long long nonempty = 0, high = 0, mx = 0;
  for (int base = 0; base < n; base += 1024) {
    const int i = base + tid;
    const uint32_t c = i < n ? ws.bin_count[i] : 0u;
    if (i < n) {
      nonempty += c > 0;
      high += c >= (uint32_t)kSortSmemCap;
      mx = c > mx ? c : mx;
      // one shared-memory atomic per warp and size class (most bins of a warp share one)
      const uint32_t cls = c ? 33 - __clz(c) : 0;
      const unsigned act = __activemask();
      const unsigned peers = __match_any_sync(act, cls);
      if (lane == __ffs(peers) - 1) atomicAdd(&cls_count[cls], (uint32_t)__popc(peers));
    }
    unsigned long long x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      unsigned long long s = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    const unsigned long long incl = x + (wid ? warp_sums[wid - 1] : 0ull) + carry;
    if (i < n) {
      const unsigned long long excl = incl - c;
      ws.bin_off[i] = (uint32_t)min(excl, (unsigned long long)ws.refs_cap);
      ws.bin_cursor[i] = (uint32_t)min(excl, (unsigned long long)ws.refs_cap);
    }
    __syncthreads();
    if (tid == 1023) carry = incl;
    __syncthreads();
  }
  if (tid == 0) {
    ws.bin_off[n] = (uint32_t)min(carry, (unsigned long long)ws.refs_cap);
    ws.ctrl->refs_total = carry;
    ws.ctrl->raster_items = (unsigned long long)n * bin_hb(ws.bin_log2);
    if (carry > (unsigned long long)ws.refs_cap) set_error(ws.ctrl, LR_ERR_OVERFLOW);
  }
  // statistics
  for (int o = 16; o > 0; o >>= 1) {
    nonempty += __shfl_xor_sync(0xffffffffu, nonempty, o);
    high += __shfl_xor_sync(0xffffffffu, high, o);
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if (lane == 0) {
    atomicAdd(&ws.ctrl->bins_nonempty, nonempty);
    atomicAdd(&ws.ctrl->bins_high, high);
    atomicMax(&ws.ctrl->max_bin, mx);
  }
  __syncthreads();
  // class bases, largest class first
  if (tid == 0) {
    uint32_t s = 0;
    for (int k = 33; k >= 0; --k) { cls_base[k] = s; s += cls_count[k]; }
  }
  __syncthreads();
  for (int i = tid; i < n; i += 1024) {
    const uint32_t c = ws.bin_count[i];
    const uint32_t cls = c ? 33 - __clz(c) : 0;
    // lanes of one class take consecutive positions from one atomic of their leader
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, cls);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&cls_base[cls], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    ws.bin_order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

__global__ __launch_bounds__(kBinThreads, kBinMinBlocks) void k_bin_scatter(Ws ws) {
  pdl_begin();
  __shared__ uint32_t hist[kHistSmemBins];
  if (ws.ctrl->error == LR_ERR_OVERFLOW) return;
  const int v = view_of_chunk(ws.views, ws.n_views, blockIdx.x);
  const ViewDev& V = ws.views[v];
  const long long q0 = V.quad_base + (long long)(blockIdx.x - V.chunk_base) * kChunkQuads;
  const long long q1 = min(q0 + kChunkQuads, V.quad_base + V.num_quads);
  const int nb = V.nbx * V.nby;
  const bool smem = nb <= kHistSmemBins;
  if (smem) {
    // the chunk's range in each bin it touches, reserved by k_bin_count
    const uint2 sp = ws.chunk_span[blockIdx.x];
    const uint2* list = reinterpret_cast<const uint2*>(ws.refs_tmp) + sp.x;
    for (int i = threadIdx.x; i < (int)sp.y; i += blockDim.x) {
      const uint2 e = list[i];
      hist[e.x] = ws.bin_off[V.bin_base + e.x] + e.y;
    }
    __syncthreads();
  }
  for_each_ref<false>(ws, V, q0, q1, [&](long long q, int b, int bx, int by, uint2 rect, uint32_t info) {
    const uint32_t slot = smem ? atomicAdd(&hist[b], 1u) : atomicAdd(&ws.bin_cursor[V.bin_base + b], 1u);
    const int lg = ws.bin_log2;
    const int x0 = max((int)(rect.x & 0xffff), bx << lg);
    const int x1 = min((int)(rect.x >> 16), ((bx + 1) << lg) - 1);
    const int y0 = max((int)(rect.y & 0xffff), by << lg);
    const int y1 = min((int)(rect.y >> 16), ((by + 1) << lg) - 1);
    // a quad inside one bin, or of constant depth: its per-quad value; else the plane at its
    // box clipped to this bin
    const bool one_bin = ((rect.x & 0xffff) >> lg) == ((rect.x >> 16) >> lg) &&
                         ((rect.y & 0xffff) >> lg) == ((rect.y >> 16) >> lg);
    const float rep = (one_bin || (info & kInfoFlatDepth)) ? ws.rec_rep[q] : rep_depth(ws, q, info, x0, x1, y0, y1);
    if (slot < (uint32_t)ws.refs_cap) ws.refs[slot] = ref_key(rep, q);
  });
}


// Merge sorted runs a[0, na) and b[0, nb) into out, split evenly over the CTA (merge path).
__device__ void cta_merge(const unsigned long long* a, int na, const unsigned long long* b, int nb,
                          unsigned long long* out) {
  const int total = na + nb;
  const int per = (total + blockDim.x - 1) / blockDim.x;
  const int d0 = min((int)threadIdx.x * per, total), d1 = min(d0 + per, total);
  if (d0 >= d1) return;
  // find i + j = d0 with a[i-1] < b[j] and b[j-1] < a[i] (keys are unique)
  int lo = max(0, d0 - nb), hi = min(d0, na);
  while (lo < hi) {
    const int i = (lo + hi) >> 1;
    if (a[i] < b[d0 - i - 1]) lo = i + 1; else hi = i;
  }
  int i = lo, j = d0 - lo;
  for (int d = d0; d < d1; ++d) {
    if (j >= nb || (i < na && a[i] < b[j])) out[d] = a[i++];
    else out[d] = b[j++];
  }
}

// The bin's transposed half-block bitmap (hb_row): for each sorted reference, the mask of
// the bin's 8x4 half-blocks (bit hy * cols + hx, in mw 32-bit words) that the quad's pixel
// AABB overlaps, computed one warp per 32 references and transposed across the warp word by
// word, so that row h, word w holds the bits of references 32 w .. 32 w + 31 for half-block
// h. The rasteriser then reads a half-block's candidates with one coalesced load per 1024
// references. When the bitmap fits `stage` (shared memory, stage_words 32-bit words), the
// transposed words are assembled there and copied out row by row with coalesced stores;
// otherwise each lane stores its word of a row directly.
__device__ void write_hb_bitmap(const Ws& ws, const unsigned long long* r, int n, int bin, uint32_t* stage,
                                int stage_words) {
  const int v = view_of_bin(ws.views, ws.n_views, bin);
  const ViewDev& V = ws.views[v];
  const int b = bin - V.bin_base;
  const int lg = ws.bin_log2, B = 1 << lg;
  const int cols = bin_hb_cols(lg), mw = bin_mw(lg), mrows = bin_mrows(lg);
  const int rpw = 32 / cols;                              // half-block rows per mask word
  // bit i * cols for every row i of a word: the row pattern's replication
  const uint32_t rep = cols == 8 ? 0x01010101u : (cols == 4 ? 0x11111111u : 0x55555555u);
  const int x0 = (b % V.nbx) << lg, y0 = (b / V.nbx) << lg;
  const int nw = (n + 31) >> 5;
  const int lane = threadIdx.x & 31;
  uint32_t* bm = ws.ref_hb + (size_t)mw * (size_t)(r - ws.refs) + (size_t)mrows * (size_t)bin;
  const bool staged = mrows * nw <= stage_words;
  uint32_t* dst = staged ? stage : bm;
  for (int w = threadIdx.x >> 5; w < nw; w += blockDim.x >> 5) {
    const int i = 32 * w + lane;
    int hx0 = 1, hx1 = 0, hy0 = 1, hy1 = 0;                // empty unless the box meets the bin
    const uint32_t rec = i < n ? ~(uint32_t)r[i] : 0xFFFFFFFFu;
    if (rec < (uint64_t)ws.total_quads) {
      const uint2 rc = ws.rec_rect[rec];
      const int px0 = max((int)(rc.x & 0xffff), x0) - x0, px1 = min((int)(rc.x >> 16), x0 + B - 1) - x0;
      const int py0 = max((int)(rc.y & 0xffff), y0) - y0, py1 = min((int)(rc.y >> 16), y0 + B - 1) - y0;
      if (px0 <= px1 && py0 <= py1) {
        hx0 = px0 / kHbW; hx1 = px1 / kHbW; hy0 = py0 / kHbH; hy1 = py1 / kHbH;
      }
    }
    // the half-block columns hx0..hx1 replicated into the rows hy0..hy1 that fall in mask
    // word m: a product, since a row's pattern never carries into the next row
    const uint32_t row = hx0 <= hx1 ? ((2u << hx1) - 1u) & ~((1u << hx0) - 1u) : 0u;
    for (int m = 0; m < mw; ++m) {
      const int a = max(hy0 - m * rpw, 0), c = min(hy1 - m * rpw, rpw - 1);
      const uint32_t rows = a <= c ? rep & ((2u << (c * cols)) - 1u) & ~((1u << (a * cols)) - 1u) : 0u;
      dst[(size_t)(32 * m + lane) * nw + w] = warp_transpose32(row * rows, lane);
    }
  }
  if (staged) {
    __syncthreads();
    for (int i = threadIdx.x; i < mrows * nw; i += blockDim.x) bm[i] = stage[i];
  }
}

// Block-wide reduction / exclusive scan helpers over all threads of the CTA (blockDim a
// multiple of 32, at most 1024); red holds 32 words of shared scratch.
__device__ __forceinline__ uint32_t block_min_u32(uint32_t v, uint32_t* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  v = lane < nw ? red[lane] : 0xFFFFFFFFu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ uint32_t block_max_u32(uint32_t v, uint32_t* red) {
  return ~block_min_u32(~v, red);
}
// exclusive prefix sum of v over threads (in thread order); *total receives the sum
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* red, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) red[w] = incl;
  __syncthreads();
  uint32_t ws = lane < nw ? red[lane] : 0u;
  uint32_t wincl = ws;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, wincl, o);
    if (lane >= o) wincl += t;
  }
  *total = __shfl_sync(0xffffffffu, wincl, 31);
  const uint32_t wbase = __shfl_sync(0xffffffffu, wincl - ws, w);
  return wbase + incl - v;
}

// Ascending bucket sort of the 64-bit keys r[0, n) by the whole CTA, through shared memory
// dst[n] and cnt[2 * NBMAX + 2] (NBMAX a power of two). Keys are bucketed by their high word,
// linearly between its minimum and maximum over the list (monotone, so buckets come out in
// order), each bucket is sorted by insertion by one thread, and the result is written back
// to r. Returns false, with r unchanged, when a bucket would hold more than kMaxBucket keys
// (many equal or clustered depths); the caller then uses a comparison sort.
template <int NBMAX>
__device__ bool cta_bucket_sort(unsigned long long* r, int n, unsigned long long* dst, uint32_t* cnt,
                                uint32_t* red) {
  const int T = (int)blockDim.x, tid = threadIdx.x;
  // about two keys per bucket: a power of two in [32, NBMAX]
  int NB = 32;
  while (NB < NBMAX && 2 * NB < n) NB <<= 1;
  uint32_t lo = 0xFFFFFFFFu, hi = 0u;
  for (int i = tid; i < n; i += T) {
    const uint32_t h = (uint32_t)(r[i] >> 32);
    lo = min(lo, h);
    hi = max(hi, h);
  }
  lo = block_min_u32(lo, red);
  hi = block_max_u32(hi, red);
  const float scale = (float)NB / ((float)(hi - lo) + 1.0f);
  auto bucket = [&](unsigned long long key) {
    return min(NB - 1, (int)((float)((uint32_t)(key >> 32) - lo) * scale));
  };
  uint32_t* start = cnt;            // [NB + 1]
  uint32_t* cur = cnt + NBMAX + 1;  // [NB]
  for (int b = tid; b < NB; b += T) start[b] = 0u;
  __syncthreads();
  for (int i = tid; i < n; i += T) atomicAdd(&start[bucket(r[i])], 1u);
  __syncthreads();
  // each thread owns `per` consecutive buckets (threads past NB own none): the largest
  // bucket and the buckets' sum
  const int per = NB >= T ? NB / T : 1;
  const int mine = tid * per < NB ? per : 0;
  uint32_t mx = 0u, sum = 0u;
  for (int k = 0; k < mine; ++k) {
    const uint32_t c = start[tid * per + k];
    mx = max(mx, c);
    sum += c;
  }
  mx = block_max_u32(mx, red);
  if (mx > (uint32_t)kMaxBucket) return false;
  uint32_t total = 0;
  uint32_t base = block_excl_scan(sum, red, &total);
  __syncthreads();
  for (int k = 0; k < mine; ++k) {
    const int b = tid * per + k;
    const uint32_t c = start[b];
    start[b] = base;
    cur[b] = base;
    base += c;
  }
  if (tid == 0) start[NB] = (uint32_t)n;
  __syncthreads();
  for (int i = tid; i < n; i += T) {
    const unsigned long long key = r[i];
    dst[atomicAdd(&cur[bucket(key)], 1u)] = key;
  }
  __syncthreads();
  for (int b = tid; b < NB; b += T) {
    const int s0 = (int)start[b], s1 = (int)start[b + 1];
    for (int i = s0 + 1; i < s1; ++i) {
      const unsigned long long x = dst[i];
      int j = i - 1;
      while (j >= s0 && dst[j] > x) {
        dst[j + 1] = dst[j];
        --j;
      }
      dst[j + 1] = x;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += T) r[i] = dst[i];
  __syncthreads();
  return true;
}

// Ascending sort of the 32 KPL keys v (KPL per lane, lane l holding elements KPL l ..
// KPL l + KPL - 1) by one warp: a bitonic network, its compare-exchanges between a lane's own
// keys (element distance below KPL) in registers and the others by shuffles with the
// partner lane.
template <int KPL>
__device__ __forceinline__ void warp_bitonic(unsigned long long v[KPL], int lane) {
#pragma unroll
  for (int k = 2; k <= 32 * KPL; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < KPL) {
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
          if (r & j) continue;   // r is the lower element of the pair (r, r + j)
          // ascending where element KPL lane + r has bit k clear
          const bool asc = k < KPL ? (r & k) == 0 : (lane & (k / KPL)) == 0;
          const unsigned long long a = v[r], b = v[r | j];
          const bool sw = asc ? (a > b) : (a < b);
          v[r] = sw ? b : a;
          v[r | j] = sw ? a : b;
        }
      } else {
        const int lj = j / KPL;
        const bool asc = (lane & (k / KPL)) == 0;
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
          const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[r], lj);
          // the lower element of an ascending pair (or the upper of a descending one) keeps
          // the smaller key
          v[r] = (asc == lower) ? (v[r] < o ? v[r] : o) : (v[r] > o ? v[r] : o);
        }
      }
    }
  }
}

// Runs of 32 KPL keys of g[0, n), one warp each, sorted into A (padded with the largest key
// up to the end of the last run).
template <int KPL>
__device__ __forceinline__ void sort_runs(const unsigned long long* g, int n, unsigned long long* A) {
  constexpr int L = 32 * KPL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; L * r < n; r += nw) {
    unsigned long long v[KPL];
    const int base = L * r + KPL * lane;
#pragma unroll
    for (int k = 0; k < KPL; ++k) v[k] = base + k < n ? g[base + k] : ~0ull;
    warp_bitonic<KPL>(v, lane);
#pragma unroll
    for (int k = 0; k < KPL; ++k) A[base + k] = v[k];
  }
}

// Ascending merge sort of g[0, n) (n <= 256 * warps of the CTA) in shared memory by the whole
// CTA: runs sorted in registers, one per warp (sort_runs), then merge levels between two
// shared buffers, each thread producing an equal slice of every level's output (merge path
// search + a sequential merge of its slice). Runs are 256 keys long when nearly every warp
// gets one, else 128 or 64 (a warp without a run would wait at the barrier). The keys are
// padded to a power of two N with the largest key, so every output position from n on
// holds padding at every level: both buffers are padded once, and the runs and output
// slices starting at n or later are skipped.
__device__ __forceinline__ void cta_merge_sort_smem(unsigned long long* g, int n, unsigned long long* A,
                                    unsigned long long* Bf) {
  const int T = (int)blockDim.x, t = threadIdx.x, nw = T >> 5;
  const int run = n > (nw - 1) * 256 ? 256 : (n > (nw - 1) * 128 ? 128 : 64);
  int N = run;
  while (N < n) N <<= 1;
  if (run == 256) sort_runs<8>(g, n, A);
  else if (run == 128) sort_runs<4>(g, n, A);
  else sort_runs<2>(g, n, A);
  for (int i = ((n + run - 1) / run) * run + t; i < N; i += T) A[i] = ~0ull;
  for (int i = n + t; i < N; i += T) Bf[i] = ~0ull;
  __syncthreads();
  unsigned long long* src = A;
  unsigned long long* dst = Bf;
  for (int w = run; w < N; w <<= 1) {
    const int P = N / T > 0 ? N / T : 1;      // outputs per thread; divides 2w
    for (int d0 = t * P; d0 < n; d0 += T * P) {
      const int base = (d0 / (2 * w)) * (2 * w), loc = d0 - base;
      const unsigned long long* a = src + base;
      const unsigned long long* b = src + base + w;
      int lo = max(0, loc - w), hi = min(loc, w);
      while (lo < hi) {
        const int i = (lo + hi) >> 1;
        if (a[i] < b[loc - i - 1]) lo = i + 1; else hi = i;
      }
      int i = lo, j = loc - lo;
      for (int d = 0; d < P; ++d) {
        const bool ta = j >= w || (i < w && a[i] < b[j]);
        dst[base + loc + d] = ta ? a[i] : b[j];
        i += ta;
        j += !ta;
      }
    }
    __syncthreads();
    unsigned long long* tmp = src; src = dst; dst = tmp;
  }
  for (int i = t; i < n; i += T) g[i] = src[i];
}

// Whether a bin is rasterised by this render: with an owned-tile set, whether any 32x32-pixel
// tile the bin covers is owned (a bin of 16 pixels lies in one tile, one of 64 spans up to
// four).
__device__ __forceinline__ bool bin_owned(const Ws& ws, int bin) {
  const int v = view_of_bin(ws.views, ws.n_views, bin);
  const ViewDev& V = ws.views[v];
  if (!V.owned) return true;
  const int b = bin - V.bin_base, lg = ws.bin_log2;
  const int x0 = (b % V.nbx) << lg, y0 = (b / V.nbx) << lg;
  const int x1 = min(x0 + (1 << lg), V.width) - 1, y1 = min(y0 + (1 << lg), V.height) - 1;
  for (int ty = y0 >> kTileLog2; ty <= (y1 >> kTileLog2); ++ty)
    for (int tx = x0 >> kTileLog2; tx <= (x1 >> kTileLog2); ++tx)
      if (tile_owned(V, tx << kTileLog2, ty << kTileLog2)) return true;
  return false;
}

#ifndef LR_SORT_MIN_BLOCKS
#define LR_SORT_MIN_BLOCKS 5   // resident CTAs per SM (48 registers, no spills)
#endif
__global__ __launch_bounds__(256, LR_SORT_MIN_BLOCKS) void k_bin_sort(Ws ws) {
  pdl_begin();
  extern __shared__ unsigned long long sbuf[];
  if (ws.ctrl->error == LR_ERR_OVERFLOW) return;
  const int bin = blockIdx.x;
  const uint32_t off = ws.bin_off[bin];
  const int n = (int)(ws.bin_off[bin + 1] - off);
  if (n >= kSortSmemCap) return;   // high-density: k_bin_sort_big
  if (!bin_owned(ws, bin)) return;  // a tile another renderer rasterises
  unsigned long long* r = ws.refs + off;
  if (n > 1) {
    cta_merge_sort_smem(r, n, sbuf, sbuf + kSortSmemCap);
    __syncthreads();
  }
  write_hb_bitmap(ws, r, n, bin, reinterpret_cast<uint32_t*>(sbuf), (int)(kSortSmemBytes / 4));
}

__global__ __launch_bounds__(kSortBigThreads, 1) void k_bin_sort_big(Ws ws) {
  pdl_begin();
  extern __shared__ unsigned long long sbuf[];
  __shared__ int s_bin;
  if (ws.ctrl->error == LR_ERR_OVERFLOW) return;
  const unsigned long long n_big = ws.ctrl->bins_high;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long k = atomicAdd(&ws.ctrl->sort_head, 1ull);
      s_bin = k < n_big ? (int)ws.bin_order[k] : -1;
    }
    __syncthreads();
    const int bin = s_bin;
    __syncthreads();
    if (bin < 0) return;
    if (!bin_owned(ws, bin)) continue;
    const uint32_t off = ws.bin_off[bin];
    const int n = (int)(ws.bin_off[bin + 1] - off);
    unsigned long long* r = ws.refs + off;
    __shared__ uint32_t red[32];
    if (n <= kBucketBigCap &&
        cta_bucket_sort<kBucketsBig>(r, n, sbuf, reinterpret_cast<uint32_t*>(sbuf + kBucketBigCap), red)) {
      if (threadIdx.x == 0) atomicAdd(&ws.ctrl->sort_branch[0], 1ull);
      write_hb_bitmap(ws, r, n, bin, reinterpret_cast<uint32_t*>(sbuf), (int)(kSortBigSmemBytes / 4));
      __syncthreads();
      continue;
    }
    const int run0 = n <= kSortBigCap ? n : kSortBigCap;
    if (threadIdx.x == 0) atomicAdd(&ws.ctrl->sort_branch[n <= kSortBigCap ? 1 : 2], 1ull);
    // sort runs of up to kSortBigCap references in shared memory
    for (int s = 0; s < n; s += run0) {
      cta_merge_sort_smem(r + s, min(run0, n - s), sbuf, sbuf + kSortBigCap);
      __syncthreads();
    }
    // merge the runs through the global buffer (only for more than kSortBigCap)
    unsigned long long* src = r;
    unsigned long long* dst = ws.refs_tmp + off;
    for (int run = run0; run < n; run <<= 1) {
      for (int s = 0; s < n; s += 2 * run) {
        const int na = min(run, n - s);
        const int nbb = min(run, max(0, n - s - run));
        cta_merge(src + s, na, src + s + na, nbb, dst + s);
      }
      __syncthreads();
      unsigned long long* t = src; src = dst; dst = t;
    }
    if (src != r) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = src[i];
    }
    __syncthreads();
    write_hb_bitmap(ws, r, n, bin, reinterpret_cast<uint32_t*>(sbuf), (int)(kSortBigSmemBytes / 4));
    __syncthreads();
  }
}

}  // namespace lr
