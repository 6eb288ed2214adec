// lr_raster8.cuh -- the bin rasteriser with 8x8-pixel blocks as work items, the other block
// shape of the autotuner (lr_config.block_h = 8). The paper sorts tri-blocks per 8x8 block
// (Sec. 2, Stage 3, Phase 2) and rasterises tri-half-blocks of 8x4 (Phase 3); lr_raster.cuh
// takes the 8x4 half-block as the work item, this kernel the 8x8 block.
//
// One warp takes one block, i.e. two vertically stacked half-blocks of a bin; lane L owns
// pixel (L % 8, L / 8) of the upper half and (L % 8, L / 8 + 4) of the lower one. The
// candidates are the quads whose pixel box meets either half (the union of the two
// half-blocks' bitmap rows, in sorted order), each set up once for the block, so a quad
// that covers both halves is set up once instead of twice. Per round of 32 candidates every
// lane computes its quad's two triangles' coverage masks for both halves; after the
// transposes the two halves' pixels run the fragment loop one after the other. Between
// rounds each lane's two per-pixel sorter states are parked in shared memory, so only one
// is live in registers. Everything else (exact depth key, K-slot sorter, misorder
// detection, blending, the exact path for flagged pixels) is the 8x4 rasteriser's.
// Forward exact renders with flat or per-vertex colours and K <= 3 only; other renders use
// the 8x4 kernel (the image is the same either way).
#pragma once

#include "lr_raster.cuh"

namespace lr {

constexpr int kBlkH = 8;          // rows of the block work item

// Coverage of the block's 64 pixel centres (bit ly * 8 + lx) by a triangle that needs
// exact 64-bit edge values, pixel by pixel.
static __device__ __noinline__ unsigned long long tri_mask_slow8(const TriSm& T, int ox, int oy, const int box[4]) {
  unsigned long long mask = 0;
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
      if (cov) mask |= 1ull << (ly * kHbW + lx);
    }
  return mask;
}

// One pixel's sorter state and counters while the lane works on its other pixel.
template <int K, bool VTX>
struct Parked {
  static constexpr int kCols = (VTX || PixelState<K, VTX>::kPrefetch) ? K : 1;
  float4 c[kCols];
  unsigned long long s[K];
  unsigned long long last;
  unsigned long long hsh;
  float r, g, b, T;
  uint32_t flagged, cnt;
};

template <int K, bool VTX>
__device__ __forceinline__ void park(Parked<K, VTX>& P, const PixelState<K, VTX>& st, uint32_t cnt,
                                     unsigned long long hsh) {
#pragma unroll
  for (int i = 0; i < K; ++i) P.s[i] = st.s[i];
#pragma unroll
  for (int i = 0; i < Parked<K, VTX>::kCols; ++i) P.c[i] = st.c[i];
  P.last = st.last;
  P.r = st.r; P.g = st.g; P.b = st.b; P.T = st.T;
  P.flagged = st.flagged;
  P.cnt = cnt;
  P.hsh = hsh;
}

template <int K, bool VTX>
__device__ __forceinline__ void unpark(const Parked<K, VTX>& P, PixelState<K, VTX>& st, uint32_t& cnt,
                                       unsigned long long& hsh) {
#pragma unroll
  for (int i = 0; i < K; ++i) st.s[i] = P.s[i];
#pragma unroll
  for (int i = 0; i < Parked<K, VTX>::kCols; ++i) st.c[i] = P.c[i];
  st.last = P.last;
  st.r = P.r; st.g = P.g; st.b = P.b; st.T = P.T;
  st.flagged = P.flagged != 0;
  cnt = P.cnt;
  hsh = P.hsh;
}

// dynamic shared memory of k_raster8: per warp 64 triangle records, 3 colour slots per
// triangle when fragments carry colours, and two parked states per lane
__host__ __device__ constexpr size_t raster8_smem_bytes(int k_sizeof_parked, bool vtx) {
  return (size_t)kRasterWarps * 64 * sizeof(TriSm) + (vtx ? (size_t)kRasterWarps * 64 * 3 * sizeof(float4) : 0) +
         (size_t)kRasterWarps * 64 * (size_t)k_sizeof_parked;
}

template <int K, bool VTX, bool HASH>
__global__ __launch_bounds__(kRasterThreads, 2) void k_raster8(Ws ws) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem[];
  using Park = Parked<K, VTX>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = lane & (kHbW - 1), ly = lane >> 3;
  TriSm* tris = reinterpret_cast<TriSm*>(smem) + warp * 64;
  float4* qcs = reinterpret_cast<float4*>(smem + (size_t)kRasterWarps * 64 * sizeof(TriSm)) + (size_t)warp * 64 * 3;
  Park* parked = reinterpret_cast<Park*>(smem + (size_t)kRasterWarps * 64 * sizeof(TriSm) +
                                         (VTX ? (size_t)kRasterWarps * 64 * 3 * sizeof(float4) : 0)) +
                 (size_t)warp * 64;
  if (ws.ctrl->error == LR_ERR_OVERFLOW) return;
  const unsigned long long nitems = ws.ctrl->raster_items >> 1;   // two half-blocks per block
  unsigned long long frag_total = 0;

  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&ws.ctrl->raster_head, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    // blocks of a bin: cols per row, rows / 2 rows; the block's half-blocks hb_u, hb_u + cols
    const int lg = ws.bin_log2, bl = bin_hb_log2(lg) - 1, cl = bin_hb_cols_log2(lg);
    const int bin_g = (int)ws.bin_order[item >> bl];
    const int blk = (int)(item & ((1u << bl) - 1u));
    const int hx = blk & ((1 << cl) - 1), hy2 = blk >> cl;
    const int hb_u = ((2 * hy2) << cl) + hx, hb_l = hb_u + (1 << cl);
    const int v = view_of_bin(ws.views, ws.n_views, bin_g);
    const ViewDev& V = ws.views[v];
    const int b = bin_g - V.bin_base;
    const int bx = b % V.nbx, by = b / V.nbx;
    const int ox = (bx << lg) + hx * kHbW, oy = (by << lg) + hy2 * kBlkH;
    if (ox >= V.width || oy >= V.height || !tile_owned(V, ox, oy)) continue;
    const int px = ox + lx;
    const bool ok0 = px < V.width && oy + ly < V.height, ok1 = px < V.width && oy + ly + kHbH < V.height;
    const uint32_t off = ws.bin_off[bin_g];
    const int n = (int)(ws.bin_off[bin_g + 1] - off);
    const bool vtx_view = V.color_mode != LR_COLOR_FLAT;
    const bool hashing = HASH && V.hash != nullptr;
    {
      PixelState<K, VTX> st;
      st.init();
      park(parked[lane], st, 0u, 0ull);
      park(parked[32 + lane], st, 0u, 0ull);
    }
    __syncwarp();

    auto process = [&](int nc, uint32_t rec) {
      // ---- triangle setup and coverage masks of both halves, one quad per lane -----------
      uint32_t tu0 = 0, tl0 = 0, tu1 = 0, tl1 = 0;
      if (lane < nc) {
        const QuadRec R = load_rec(ws.rec, rec);
        const uint32_t jl = (uint32_t)(rec - V.quad_base);
        uint32_t vsel = 0;   // per set-up triangle t: bit 8 + t, and its corners 1, 2 at bits 4t
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          TriSm& T = tris[2 * lane + t];
          int cor[3];
          uint32_t mu, ml;
          if (R.info & (kInfoSmall0 << t)) {
            int box[4], le[3], lsx[3], lsy[3];
            if (!setup_tri_small<kBlkH>(T, R.X, R.Y, R.q, t ? R.inv[1] : R.inv[0], R.info, t, jl, ox, oy, cor, box,
                                        le, lsx, lsy))
              continue;
            // upper half: rows 0..3 of the box; lower half: the block's rows 4..7 as rows
            // 0..3 of a half-block whose edge values start four rows down
            const int bu[4] = {box[0], box[1], box[2], min(box[3], kHbH - 1)};
            const int bd[4] = {box[0], box[1], max(box[2], kHbH) - kHbH, box[3] - kHbH};
            int ld[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) ld[k] = (int)((uint32_t)le[k] + (uint32_t)kHbH * (uint32_t)lsy[k]);
            mu = tri_mask_fast(le, lsx, lsy, bu);
            ml = tri_mask_fast(ld, lsx, lsy, bd);
          } else {
            const QuadRec G = R;   // the out-of-line path's own copy (its address escapes)
            int cg[3], box[4], le[3], lsx[3], lsy[3];
            if (!setup_tri<kBlkH>(T, G.X, G.Y, G.q, G.info, t, jl, ox, oy, cg, box, le, lsx, lsy)) continue;
            if ((uint32_t)T.eb.z & kTriFast) {
              const int bu[4] = {box[0], box[1], box[2], min(box[3], kHbH - 1)};
              const int bd[4] = {box[0], box[1], max(box[2], kHbH) - kHbH, box[3] - kHbH};
              int ld[3];
#pragma unroll
              for (int k = 0; k < 3; ++k) ld[k] = (int)((uint32_t)le[k] + (uint32_t)kHbH * (uint32_t)lsy[k]);
              mu = tri_mask_fast(le, lsx, lsy, bu);
              ml = tri_mask_fast(ld, lsx, lsy, bd);
            } else {
              const unsigned long long m64 = tri_mask_slow8(T, ox, oy, box);
              mu = (uint32_t)m64;
              ml = (uint32_t)(m64 >> 32);
            }
            cor[0] = cg[0]; cor[1] = cg[1]; cor[2] = cg[2];
          }
          if (t == 0) { tu0 = mu; tl0 = ml; } else { tu1 = mu; tl1 = ml; }
          if (VTX) vsel |= (1u << (8 + t)) | ((uint32_t)(cor[1] | (cor[2] << 2)) << (4 * t));
        }
        if (VTX && vsel) {
          if (!vtx_view) {
            const float4 fc = __ldg(reinterpret_cast<const float4*>(V.col) + jl);
#pragma unroll
            for (int t = 0; t < 2; ++t)
              if (vsel & (1u << (8 + t))) {
                qcs[(2 * lane + t) * 3] = fc;
                tris[2 * lane + t].eb.z |= (int)kTriFlatCol;
              }
          } else {
            // the quad's four corner colours times 1/w; each triangle stores (c0, c1 - c0,
            // c2 - c0) of its corners for the fragment's c0 + l1 (c1 - c0) + l2 (c2 - c0)
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
              float4* qc = qcs + (2 * lane + t) * 3;
              qc[0] = p0;
              qc[1] = make_float4(a1.x - p0.x, a1.y - p0.y, a1.z - p0.z, a1.w - p0.w);
              qc[2] = make_float4(a2.x - p0.x, a2.y - p0.y, a2.z - p0.z, a2.w - p0.w);
            }
          }
        }
      }
      __syncwarp();
      // ---- transpose: lane = pixel, bit c = covered by triangle t of quad c -------------
      uint32_t mm[2][2];
      mm[0][0] = warp_transpose32(tu0, lane);
      mm[0][1] = warp_transpose32(tu1, lane);
      mm[1][0] = warp_transpose32(tl0, lane);
      mm[1][1] = warp_transpose32(tl1, lane);
      // ---- the two pixels' fragments through the K-slot sorter, one after the other --------
#pragma unroll 1
      for (int p = 0; p < 2; ++p) {
        uint32_t m0 = mm[p][0], m1 = mm[p][1];
        if (!(p ? ok1 : ok0)) m0 = m1 = 0;
        if (!__any_sync(0xffffffffu, m0 | m1)) continue;
        const int lyp = ly + p * kHbH, py = oy + lyp;
        PixelState<K, VTX> st;
        uint32_t cnt;
        unsigned long long hsh;
        unpark(parked[32 * p + lane], st, cnt, hsh);
        st.gp.grad = nullptr;
        cnt += __popc(m0) + __popc(m1);
        auto frag_step = [&]() {
          const int c = __ffs(m0 | m1) - 1;
          const uint32_t cb = 1u << c;
          const int t = (m0 & cb) ? 0 : 1;
          if (t == 0) m0 &= ~cb; else m1 &= ~cb;
          const TriSm& T = tris[2 * c + t];
          const int4 eb = T.eb;
          const uint32_t fl = (uint32_t)eb.z, id = (uint32_t)eb.w;
          if (hashing) hsh += splitmix64(id);
          if (!st.flagged) {
            const float4 kq = T.kq;
            float l1 = 0.f, l2 = 0.f;
            const float key = (!VTX && (fl & kTriConstKey)) ? kq.x : tri_key(T, T.ea, eb, kq, lx, lyp, px, py, l1, l2);
            const unsigned long long sk = ((unsigned long long)__float_as_uint(key) << 32) | id;
            float4 col = make_float4(0.f, 0.f, 0.f, 0.f);
            if (VTX) {
              const float4* qc = qcs + (2 * c + t) * 3;
              if (fl & kTriFlatCol) {
                col = qc[0];
              } else {
                const float rk = rcp_approx(key);
                const float4 a0 = qc[0], d1 = qc[1], d2 = qc[2];
                col.x = (a0.x + l1 * d1.x + l2 * d2.x) * rk;
                col.y = (a0.y + l1 * d1.y + l2 * d2.y) * rk;
                col.z = (a0.z + l1 * d1.z + l2 * d2.z) * rk;
                col.w = (a0.w + l1 * d1.w + l2 * d2.w) * rk;
              }
            }
            st.insert(sk, col, V);
          }
        };
        while (m0 | m1) frag_step();
        park(parked[32 * p + lane], st, cnt, hsh);
      }
      __syncwarp();
    };

    // ---- the block's candidates: set bits of either half's bitmap row, in sorted order --
    const uint32_t* row_u = hb_row(ws, off, bin_g, n, hb_u);
    const uint32_t* row_l = hb_row(ws, off, bin_g, n, hb_l);
    const int nw = (n + 31) >> 5;
    const uint32_t* ref_lo = reinterpret_cast<const uint32_t*>(ws.refs + off);   // low words
    for (int g = 0; g < nw; g += 32) {
      BitRounds br;
      br.prepare(g + lane < nw ? (__ldg(row_u + g + lane) | __ldg(row_l + g + lane)) : 0u, lane);
      for (int r0 = 0; r0 < br.total; r0 += 32) {
        const int j = br.get(r0, lane);
        process(min(32, br.total - r0), j < 0 ? 0u : ~ref_lo[2 * (32 * g + j)]);
      }
    }

    // ---- finish both halves ----------------------------------------------------------------
#pragma unroll 1
    for (int p = 0; p < 2; ++p) {
      PixelState<K, VTX> st;
      uint32_t cnt;
      unsigned long long hsh;
      unpark(parked[32 * p + lane], st, cnt, hsh);
      const bool ok = p ? ok1 : ok0;
      const int py = oy + ly + p * kHbH;
      if (V.xmask && oy + p * kHbH < V.height) {
        const uint32_t fm = __ballot_sync(0xffffffffu, ok && st.flagged);
        if (lane == 0) {
          const uint32_t hbw = ((uint32_t)V.width + kHbW - 1) / kHbW;
          V.xmask[((uint32_t)(oy + p * kHbH) / kHbH) * hbw + (uint32_t)ox / kHbW] = fm;
        }
      }
      if (!st.flagged) st.flush(V);
      if (ok) {
        const long long pidx = (long long)py * V.width + px;
        if (V.cnt) V.cnt[pidx] = cnt;
        if (hashing) V.hash[pidx] = hsh;
        if (!st.flagged) {
          write_pixel(V, pidx, st.r, st.g, st.b, st.T);
        } else {
          const unsigned long long slot = atomicAdd(&ws.ctrl->ovf_count, 1ull);
          ws.ovf_list[slot] = (uint32_t)(V.pix_base + pidx);
        }
        frag_total += cnt;
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) frag_total += __shfl_xor_sync(0xffffffffu, frag_total, o);
  if (lane == 0 && frag_total) atomicAdd(&ws.ctrl->fragments, frag_total);
}

}  // namespace lr

// Each translation unit lr_raster8_k<K>.cu instantiates the 8x8-block rasteriser for one
// sorter capacity K (both colour layouts, with and without the coverage hash).
#define LR_DEFINE_RASTER8(KK)                                                                 \
  namespace lr {                                                                              \
  template <bool VTX, bool HASH>                                                              \
  static cudaError_t raster8_attr_##KK(int* blocks) {                                         \
    const size_t sm = raster8_smem_bytes((int)sizeof(Parked<KK, VTX>), VTX);                  \
    cudaError_t e = cudaFuncSetAttribute(k_raster8<KK, VTX, HASH>,                            \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
    if (e == cudaSuccess && blocks)                                                           \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_raster8<KK, VTX, HASH>,     \
                                                        kRasterThreads, sm);                  \
    return e;                                                                                 \
  }                                                                                           \
  cudaError_t prepare_raster8_##KK(int* blocks_flat, int* blocks_vtx) {                       \
    cudaError_t e = raster8_attr_##KK<false, false>(blocks_flat);                             \
    if (e == cudaSuccess) e = raster8_attr_##KK<true, false>(blocks_vtx);                     \
    if (e == cudaSuccess) e = raster8_attr_##KK<false, true>(nullptr);                        \
    if (e == cudaSuccess) e = raster8_attr_##KK<true, true>(nullptr);                         \
    return e;                                                                                 \
  }                                                                                           \
  /* mode: 0 flat colours, 1 colours in the sorter; + 4: coverage hash */                      \
  cudaError_t launch_raster8_##KK(int mode, const Ws& ws, int grid, cudaStream_t st) {        \
    const size_t sf = raster8_smem_bytes((int)sizeof(Parked<KK, false>), false);              \
    const size_t sv = raster8_smem_bytes((int)sizeof(Parked<KK, true>), true);                \
    switch (mode) {                                                                           \
      case 1: k_raster8<KK, true, false><<<grid, kRasterThreads, sv, st>>>(ws); break;        \
      case 4: k_raster8<KK, false, true><<<grid, kRasterThreads, sf, st>>>(ws); break;        \
      case 5: k_raster8<KK, true, true><<<grid, kRasterThreads, sv, st>>>(ws); break;         \
      default: k_raster8<KK, false, false><<<grid, kRasterThreads, sf, st>>>(ws); break;      \
    }                                                                                         \
    return cudaGetLastError();                                                                \
  }                                                                                           \
  }
