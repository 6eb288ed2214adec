// lr_raster_strip.cuh -- the bin rasteriser with the candidate set-up shared by a CTA
// (lr_config.shared_setup = 1; 32-pixel bins). The paper's Stage 3 gives each
// bin to a workgroup whose threads first set up the bin's triangles together and then
// rasterise its blocks (Sec. 2, Stage 3, Phases 1-3); here a CTA of 8 warps takes one 32x8
// strip of a bin (8 half-blocks, one per warp, lane = pixel as in lr_raster.cuh).
//
// The strip's candidates are the bin's sorted references whose box meets any of its eight
// half-blocks (the union of their bitmap rows), taken 256 references at a time. For each
// such window the CTA (1) forms the union's words and compacts the candidates in sorted
// order, (2) sets up every candidate triangle once for the whole strip, one thread per
// triangle -- the quad record, orientation, pixel box, depth-key coefficients relative to
// the strip's first pixel centre, and for per-vertex colours the three premultiplied
// corner colours, all into shared memory -- and (3) lets every warp take its own
// half-block's candidates from the window (its bitmap row, mapped to the compacted slots),
// compute their coverage masks from the shared vertices, and run the fragment loop of
// lr_raster.cuh on the shared records. The quad records and colour gathers, the
// latency-bound part of the per-half-block set-up, are then issued once per strip by all
// 256 threads at once instead of once per half-block by every warp.
// Forward exact renders with flat or per-vertex colours and K <= 3, 32-pixel bins only;
// other renders use the 8x4 kernel (the image is the same either way).
#pragma once

#include "lr_raster.cuh"

namespace lr {

constexpr int kStripWin = 8;                       // bitmap words (256 references) per window
constexpr int kStripCap = 32 * kStripWin;          // candidate quads per window, at most
constexpr uint32_t kTriSmall = 256u;               // 32-bit key arithmetic is exact (k_setup's flag)

// shared memory of k_raster_strip: per candidate triangle a TriSm record (its pad words hold
// the pixel box relative to the strip), 3 colour slots when fragments carry colours; the
// window's union words, their prefix counts, the compacted candidates and per warp the slots
// of the current round
__host__ __device__ constexpr size_t raster_strip_smem_bytes(bool vtx) {
  return (size_t)2 * kStripCap * sizeof(TriSm) + (vtx ? (size_t)2 * kStripCap * 3 * sizeof(float4) : 0) +
         (size_t)(kStripWin + kStripWin + 1 + kStripCap + kRasterWarps * 32 + 4) * sizeof(uint32_t);
}

template <int K, bool VTX, bool HASH>
__global__ __launch_bounds__(kRasterThreads, 3) void k_raster_strip(Ws ws) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem[];
  TriSm* S_tri = reinterpret_cast<TriSm*>(smem);
  float4* S_col = reinterpret_cast<float4*>(smem + (size_t)2 * kStripCap * sizeof(TriSm));
  uint32_t* s_or = reinterpret_cast<uint32_t*>(smem + (size_t)2 * kStripCap * sizeof(TriSm) +
                                               (VTX ? (size_t)2 * kStripCap * 3 * sizeof(float4) : 0));
  uint32_t* s_pre = s_or + kStripWin;               // [kStripWin + 1]
  uint32_t* s_cand = s_pre + kStripWin + 1;         // [kStripCap] reference index within the bin
  uint32_t* s_slot = s_cand + kStripCap;            // [kRasterWarps][32]
  uint32_t* s_item = s_slot + kRasterWarps * 32;    // [4]: item, bin or -1
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int lx = lane & (kHbW - 1), ly = lane >> 3;
  const int hx = warp & 3, hyl = warp >> 2;          // this warp's half-block in the strip
  uint32_t* my_slot = s_slot + warp * 32;
  if (ws.ctrl->error == LR_ERR_OVERFLOW) return;
  const unsigned long long nitems = ws.ctrl->raster_items >> 3;   // 8 half-blocks per strip
  unsigned long long frag_total = 0;

  for (;;) {
    if (tid == 0) {
      const unsigned long long it = atomicAdd(&ws.ctrl->raster_head, 1ull);
      s_item[0] = it < nitems ? (uint32_t)it : 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t item = s_item[0];
    __syncthreads();
    if (item == 0xFFFFFFFFu) break;
    const int bin_g = (int)ws.bin_order[item >> 2];
    const int s = (int)(item & 3u);
    const int v = view_of_bin(ws.views, ws.n_views, bin_g);
    const ViewDev& V = ws.views[v];
    const int b = bin_g - V.bin_base;
    const int sx0 = (b % V.nbx) << 5, sy0 = ((b / V.nbx) << 5) + s * 2 * kHbH;   // strip origin
    if (sx0 >= V.width || sy0 >= V.height || !tile_owned(V, sx0, sy0)) continue;   // uniform
    const int ox = sx0 + hx * kHbW, oy = sy0 + hyl * kHbH;    // this warp's half-block
    const int hb = (2 * s + hyl) * 4 + hx;
    const int px = ox + lx, py = oy + ly;
    const bool pix_ok = px < V.width && py < V.height;
    const bool warp_live = ox < V.width && oy < V.height;
    const uint32_t off = ws.bin_off[bin_g];
    const int n = (int)(ws.bin_off[bin_g + 1] - off);
    const int nw = (n + 31) >> 5;
    const bool vtx_view = V.color_mode != LR_COLOR_FLAT;
    const bool hashing = HASH && V.hash != nullptr;
    const uint32_t* ref_lo = reinterpret_cast<const uint32_t*>(ws.refs + off);   // low words
    const uint32_t* my_row = hb_row(ws, off, bin_g, n, hb);

    PixelState<K, VTX> st;
    st.init();
    st.gp.grad = nullptr;
    uint32_t cnt = 0;
    unsigned long long hsh = 0;

    for (int w0 = 0; w0 < nw; w0 += kStripWin) {
      // ---- 1. the union of the strip's eight bitmap rows over the window, compacted -----
      if (tid < 8 * kStripWin) {
        const int w = w0 + (tid >> 3);
        uint32_t x = w < nw ? __ldg(hb_row(ws, off, bin_g, n, 8 * s + (tid & 7)) + w) : 0u;
        x |= __shfl_xor_sync(0xffffffffu, x, 1);
        x |= __shfl_xor_sync(0xffffffffu, x, 2);
        x |= __shfl_xor_sync(0xffffffffu, x, 4);
        if ((tid & 7) == 0) s_or[tid >> 3] = x;
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t acc = 0;
        for (int i = 0; i < kStripWin; ++i) {
          s_pre[i] = acc;
          acc += __popc(s_or[i]);
        }
        s_pre[kStripWin] = acc;
      }
      __syncthreads();
      {
        const uint32_t wd = s_or[tid >> 5];
        if ((wd >> lane) & 1u) s_cand[s_pre[tid >> 5] + __popc(wd & ((1u << lane) - 1u))] = 32u * (w0 + (tid >> 5)) + lane;
      }
      __syncthreads();
      const int nc = (int)s_pre[kStripWin];
      // ---- 2. every candidate triangle set up once for the strip, one thread each -------
      for (int e = tid; e < 2 * nc; e += kRasterThreads) {
        const int q = e >> 1, t = e & 1;
        const uint32_t rec = ~ref_lo[2 * s_cand[q]];
        const QuadRec R = load_rec(ws.rec, rec);
        TriSm& T = S_tri[e];
        uint32_t flags = 0;
        if (R.info & (t ? kInfoTri1 : kInfoTri0)) {
          // (v0, v1, v2) of T0 or (v0, v2, v3) of T1, v1 and v2 swapped for a negative area
          int xb = t ? R.X[2] : R.X[1], yb = t ? R.Y[2] : R.Y[1];
          int xc = t ? R.X[3] : R.X[2], yc = t ? R.Y[3] : R.Y[2];
          float qb = t ? R.q[2] : R.q[1], qc = t ? R.q[3] : R.q[2];
          int ib = t ? 2 : 1, ic = t ? 3 : 2;
          if (R.info & (kInfoSwap0 << t)) {
            int ti = xb; xb = xc; xc = ti;
            ti = yb; yb = yc; yc = ti;
            const float tq = qb; qb = qc; qc = tq;
            ti = ib; ib = ic; ic = ti;
          }
          const int xa = R.X[0], ya = R.Y[0];
          const float qa = R.q[0];
          // pixel-centre box, relative to the strip, clamped to a byte each
          const int bx0 = ((min(xa, min(xb, xc)) + 127) >> 8) - sx0, bx1 = ((max(xa, max(xb, xc)) - 128) >> 8) - sx0;
          const int by0 = ((min(ya, min(yb, yc)) + 127) >> 8) - sy0, by1 = ((max(ya, max(yb, yc)) - 128) >> 8) - sy0;
          if (bx0 <= 31 && bx1 >= 0 && by0 <= 2 * kHbH - 1 && by1 >= 0 && bx0 <= bx1 && by0 <= by1) {
            const uint32_t box = (uint32_t)(max(bx0, -1) + 1) | ((uint32_t)(min(bx1, 32) + 1) << 8) |
                                 ((uint32_t)(max(by0, -1) + 1) << 16) | ((uint32_t)(min(by1, 8) + 1) << 24);
            flags = kTriValid | ((qb == qa && qc == qa) ? kTriConstKey : 0u) |
                    ((R.info & (kInfoSmall0 << t)) ? kTriSmall : 0u);
            T.X[0] = xa; T.X[1] = xb; T.X[2] = xc;
            T.Y[0] = ya; T.Y[1] = yb; T.Y[2] = yc;
            T.pad[0] = (int)box;
            T.kq = make_float4(qa, __fsub_rn(qb, qa), __fsub_rn(qc, qa), t ? R.inv[1] : R.inv[0]);
            // the key's edge values (unbiased) at the strip's first pixel centre, modulo 2^32,
            // and their steps per pixel; edges v1->v2, v2->v0, v0->v1, their owned flags
            const long long P0x = 256LL * sx0 + 128, P0y = 256LL * sy0 + 128;
            const int ux[3] = {xb, xc, xa}, uy[3] = {yb, yc, ya}, wx[3] = {xc, xa, xb}, wy[3] = {yc, ya, yb};
            int ek[3], sxk[3], syk[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const long long dx = (long long)wx[k] - ux[k], dy = (long long)wy[k] - uy[k];
              if (!(dy < 0 || (dy == 0 && dx > 0))) flags |= 1u << (3 + k);
              ek[k] = (int)(uint32_t)(unsigned long long)(dx * (P0y - uy[k]) - dy * (P0x - ux[k]));
              sxk[k] = (int)(-256 * dy);
              syk[k] = (int)(256 * dx);
            }
            if (flags & kTriSmall) flags |= kTriFast;
            T.ea = make_int4(ek[1], ek[2], sxk[1], sxk[2]);
            T.eb = make_int4(syk[1], syk[2], (int)flags, (int)(2u * (uint32_t)(rec - V.quad_base) + (uint32_t)t));
            if (VTX) {
              const uint32_t jl = (uint32_t)(rec - V.quad_base);
              float4* cs = S_col + 3 * e;
              if (!vtx_view) {
                cs[0] = __ldg(reinterpret_cast<const float4*>(V.col) + jl);
                T.eb.z |= (int)kTriFlatCol;
              } else {
                uint4 vi = make_uint4(4 * jl, 4 * jl + 1, 4 * jl + 2, 4 * jl + 3);
                if (V.idx) vi = __ldg(reinterpret_cast<const uint4*>(V.idx) + jl);
                const uint32_t vb = ib == 1 ? vi.y : (ib == 2 ? vi.z : vi.w);
                const uint32_t vc = ic == 1 ? vi.y : (ic == 2 ? vi.z : vi.w);
                const float4* cv = reinterpret_cast<const float4*>(V.col);
                const float4 c0 = __ldg(cv + vi.x), c1 = __ldg(cv + vb), c2 = __ldg(cv + vc);
                const float4 p0 = make_float4(qa * c0.x, qa * c0.y, qa * c0.z, qa * c0.w);
                const float4 p1 = make_float4(qb * c1.x, qb * c1.y, qb * c1.z, qb * c1.w);
                const float4 p2 = make_float4(qc * c2.x, qc * c2.y, qc * c2.z, qc * c2.w);
                cs[0] = p0;
                cs[1] = make_float4(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z, p1.w - p0.w);
                cs[2] = make_float4(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z, p2.w - p0.w);
              }
            }
          }
        }
        if (!flags) T.eb.z = 0;
      }
      __syncthreads();
      // ---- 3. this warp's half-block: its candidates of the window, in sorted order -------
      if (warp_live) {
        BitRounds br;
        br.prepare(lane < kStripWin && w0 + lane < nw ? __ldg(my_row + w0 + lane) : 0u, lane);
        for (int r0 = 0; r0 < br.total; r0 += 32) {
          const int j = br.get(r0, lane);
          uint32_t tm0 = 0, tm1 = 0;
          if (j >= 0) {
            const int L = j >> 5, bit = j & 31;
            const uint32_t slot = s_pre[L] + __popc(s_or[L] & ((1u << bit) - 1u));
            my_slot[lane] = slot;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              const TriSm& T = S_tri[2 * slot + t];
              const uint32_t fl = (uint32_t)T.eb.z;
              if (!(fl & kTriValid)) continue;
              // the triangle's box relative to this half-block
              const uint32_t bx = (uint32_t)T.pad[0];
              int box[4] = {(int)(bx & 255u) - 1 - hx * kHbW, (int)((bx >> 8) & 255u) - 1 - hx * kHbW,
                            (int)((bx >> 16) & 255u) - 1 - hyl * kHbH, (int)(bx >> 24) - 1 - hyl * kHbH};
              if (box[0] > kHbW - 1 || box[1] < 0 || box[2] > kHbH - 1 || box[3] < 0) continue;
              box[0] = max(box[0], 0);
              box[1] = min(box[1], kHbW - 1);
              box[2] = max(box[2], 0);
              box[3] = min(box[3], kHbH - 1);
              uint32_t mk;
              if (fl & kTriSmall) {
                // biased edge values at the half-block's first pixel centre: 32-bit exact for
                // a small triangle whose box meets the half-block
                const int P0x = 256 * ox + 128, P0y = 256 * oy + 128;
                const int ux[3] = {T.X[1], T.X[2], T.X[0]}, uy[3] = {T.Y[1], T.Y[2], T.Y[0]};
                const int wx[3] = {T.X[2], T.X[0], T.X[1]}, wy[3] = {T.Y[2], T.Y[0], T.Y[1]};
                int le[3], lsx[3], lsy[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                  const int dx = wx[k] - ux[k], dy = wy[k] - uy[k];
                  le[k] = (int)((uint32_t)dx * (uint32_t)(P0y - uy[k]) - (uint32_t)dy * (uint32_t)(P0x - ux[k])) -
                          (int)((fl >> (3 + k)) & 1u);
                  lsx[k] = -256 * dy;
                  lsy[k] = 256 * dx;
                }
                mk = tri_mask_fast(le, lsx, lsy, box);
              } else {
                mk = tri_mask_slow(T, ox, oy, box);
              }
              if (t == 0) tm0 = mk; else tm1 = mk;
            }
          }
          __syncwarp();
          // ---- transpose; fragments through the K-slot sorter ----------------------------
          uint32_t m0 = warp_transpose32(tm0, lane), m1 = warp_transpose32(tm1, lane);
          if (!pix_ok) m0 = m1 = 0;
          cnt += __popc(m0) + __popc(m1);
          const int lxs = hx * kHbW + lx, lys = hyl * kHbH + ly;   // pixel relative to the strip
          auto frag_step = [&]() {
            const int c = __ffs(m0 | m1) - 1;
            const uint32_t cb = 1u << c;
            const int t = (m0 & cb) ? 0 : 1;
            if (t == 0) m0 &= ~cb; else m1 &= ~cb;
            const uint32_t slot = my_slot[c];
            const TriSm& T = S_tri[2 * slot + t];
            const int4 eb = T.eb;
            const uint32_t fl = (uint32_t)eb.z, id = (uint32_t)eb.w;
            if (hashing) hsh += splitmix64(id);
            if (!st.flagged) {
              const float4 kq = T.kq;
              float l1 = 0.f, l2 = 0.f;
              const float key = (!VTX && (fl & kTriConstKey)) ? kq.x : tri_key(T, T.ea, eb, kq, lxs, lys, px, py, l1, l2);
              const unsigned long long sk = ((unsigned long long)__float_as_uint(key) << 32) | id;
              float4 col = make_float4(0.f, 0.f, 0.f, 0.f);
              if (VTX) {
                const float4* qc = S_col + 3 * (2 * slot + t);
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
          if (VTX) {
            while (m0 | m1) frag_step();
          } else {
            while (m0 | m1) {
              frag_step();
              if (!(m0 | m1)) break;
              frag_step();
            }
          }
          __syncwarp();
        }
      }
      __syncthreads();   // the window's records are overwritten next
    }

    // ---- finish the half-block -------------------------------------------------------------
    if (warp_live) {
      if (V.xmask) {
        const uint32_t fm = __ballot_sync(0xffffffffu, pix_ok && st.flagged);
        if (lane == 0) {
          const uint32_t hbw = ((uint32_t)V.width + kHbW - 1) / kHbW;
          V.xmask[((uint32_t)oy / kHbH) * hbw + (uint32_t)ox / kHbW] = fm;
        }
      }
      if (!st.flagged) st.flush(V);
      if (pix_ok) {
        const long long pidx = (long long)py * V.width + px;
        if (V.cnt) V.cnt[pidx] = cnt;
        if (hashing) V.hash[pidx] = hsh;
        if (!st.flagged) {
          write_pixel(V, pidx, st.r, st.g, st.b, st.T);
        } else {
          const unsigned long long slot = atomicAdd(&ws.ctrl->ovf_count, 1ull);
          ws.ovf_list[slot] = (uint32_t)(V.pix_base + pidx);
        }
      }
      frag_total += cnt;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) frag_total += __shfl_xor_sync(0xffffffffu, frag_total, o);
  if (lane == 0 && frag_total) atomicAdd(&ws.ctrl->fragments, frag_total);
}

}  // namespace lr

// Each translation unit lr_raster_strip_k<K>.cu instantiates the strip rasteriser for one
// sorter capacity K (both colour layouts, with and without the coverage hash).
#define LR_DEFINE_RASTER_STRIP(KK)                                                            \
  namespace lr {                                                                              \
  template <bool VTX, bool HASH>                                                              \
  static cudaError_t raster_strip_attr_##KK(int* blocks) {                                    \
    const size_t sm = raster_strip_smem_bytes(VTX);                                           \
    cudaError_t e = cudaFuncSetAttribute(k_raster_strip<KK, VTX, HASH>,                       \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
    if (e == cudaSuccess && blocks)                                                           \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_raster_strip<KK, VTX, HASH>, \
                                                        kRasterThreads, sm);                  \
    return e;                                                                                 \
  }                                                                                           \
  cudaError_t prepare_raster_strip_##KK(int* blocks_flat, int* blocks_vtx) {                  \
    cudaError_t e = raster_strip_attr_##KK<false, false>(blocks_flat);                        \
    if (e == cudaSuccess) e = raster_strip_attr_##KK<true, false>(blocks_vtx);                \
    if (e == cudaSuccess) e = raster_strip_attr_##KK<false, true>(nullptr);                   \
    if (e == cudaSuccess) e = raster_strip_attr_##KK<true, true>(nullptr);                    \
    return e;                                                                                 \
  }                                                                                           \
  /* mode: 0 flat colours, 1 colours in the sorter; + 4: coverage hash */                      \
  cudaError_t launch_raster_strip_##KK(int mode, const Ws& ws, int grid, cudaStream_t st) {   \
    const size_t sf = raster_strip_smem_bytes(false), sv = raster_strip_smem_bytes(true);     \
    switch (mode) {                                                                           \
      case 1: k_raster_strip<KK, true, false><<<grid, kRasterThreads, sv, st>>>(ws); break;   \
      case 4: k_raster_strip<KK, false, true><<<grid, kRasterThreads, sf, st>>>(ws); break;   \
      case 5: k_raster_strip<KK, true, true><<<grid, kRasterThreads, sv, st>>>(ws); break;    \
      default: k_raster_strip<KK, false, false><<<grid, kRasterThreads, sf, st>>>(ws); break; \
    }                                                                                         \
    return cudaGetLastError();                                                                \
  }                                                                                           \
  }
