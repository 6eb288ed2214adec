// lr_exact.cuh -- the exact path for one pixel (the per-pixel full sort the paper suggests
// for the pixels its fixed-size sorter misorders, Sec. 2, "Sample blending"), used by
// k_overflow (lr_overflow.cu) for the pixels the rasteriser registered.
//
// One warp per pixel: the candidates of the pixel's half-block from the bin's transposed
// bitmap (one coalesced load per 1024 references), their fragments re-evaluated exactly
// (the rasteriser's edge tests and depth key), sorted fully and composited front to back.
// Memory is bounded: a pass keeps the KEEP nearest fragments below a threshold in a
// shared-memory buffer (when it fills, it is sorted and cut back to KEEP), composites them,
// lowers the threshold to the last composited key and repeats until no fragment is left, so
// any depth complexity is handled at one re-scan of the candidates per KEEP fragments.
// (Running it inside the rasteriser for a half-block's few flagged pixels was measured: the
// call's registers slowed the rasteriser's fragment loop far more than it saved.)
#pragma once

#include "lr_raster.cuh"

namespace lr {

// Exact fragment of record rec, triangle t at pixel (px, py): returns false if the pixel
// centre is not covered; otherwise the sort key and (if col) the straight RGBA colour.
// The triangle's vertices are picked with selects, so the record stays in registers.
__device__ __forceinline__ bool frag_eval_r(const Ws& ws, const ViewDev& V, const QuadRec& R, uint32_t rec, int t,
                                            int px, int py, unsigned long long& sk, float4* col) {
  if (!(R.info & (t ? kInfoTri1 : kInfoTri0))) return false;
  // triangle t = (v0, v[1 + t], v[2 + t]); a negative area swaps its last two vertices
  const bool sw = (R.info & (kInfoSwap0 << t)) != 0;
  const int ib = sw ? 2 + t : 1 + t, ic = sw ? 1 + t : 2 + t;
  const int xa = R.X[0], ya = R.Y[0];
  const int xb = ib == 1 ? R.X[1] : (ib == 2 ? R.X[2] : R.X[3]);
  const int yb = ib == 1 ? R.Y[1] : (ib == 2 ? R.Y[2] : R.Y[3]);
  const int xc = ic == 1 ? R.X[1] : (ic == 2 ? R.X[2] : R.X[3]);
  const int yc = ic == 1 ? R.Y[1] : (ic == 2 ? R.Y[2] : R.Y[3]);
  // edge functions e0 = E(b -> c), e1 = E(c -> a), e2 = E(a -> b); top-left rule. A
  // covered pixel centre lies inside the triangle's vertex box, so a pixel outside the
  // triangle's pixel-centre box is not covered; inside it, a triangle k_setup marked small
  // has every edge value in (-2^30, 2^30), and 32-bit arithmetic is exact. Otherwise 64-bit.
  long long e[3];
  {
    const int ux[3] = {xb, xc, xa}, uy[3] = {yb, yc, ya}, wx[3] = {xc, xa, xb}, wy[3] = {yc, ya, yb};
    if (R.info & (kInfoSmall0 << t)) {
      if (px < ((min(xa, min(xb, xc)) + 127) >> 8) || px > ((max(xa, max(xb, xc)) - 128) >> 8) ||
          py < ((min(ya, min(yb, yc)) + 127) >> 8) || py > ((max(ya, max(yb, yc)) - 128) >> 8))
        return false;
      const int Px = 256 * px + 128, Py = 256 * py + 128;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int dx = wx[k] - ux[k], dy = wy[k] - uy[k];
        const int ek = (int)((uint32_t)dx * (uint32_t)(Py - uy[k]) - (uint32_t)dy * (uint32_t)(Px - ux[k]));
        e[k] = ek;
        const bool owned = dy < 0 || (dy == 0 && dx > 0);
        if (!(ek > 0 || (ek == 0 && owned))) return false;
      }
    } else {
      const long long Px = 256LL * px + 128, Py = 256LL * py + 128;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const long long dx = (long long)wx[k] - ux[k], dy = (long long)wy[k] - uy[k];
        e[k] = dx * (Py - uy[k]) - dy * (Px - ux[k]);
        const bool owned = dy < 0 || (dy == 0 && dx > 0);
        if (!(e[k] > 0 || (e[k] == 0 && owned))) return false;
      }
    }
  }
  const float inv = t ? R.inv[1] : R.inv[0];
  const float qa = R.q[0];
  const float qb = ib == 1 ? R.q[1] : (ib == 2 ? R.q[2] : R.q[3]);
  const float qc = ic == 1 ? R.q[1] : (ic == 2 ? R.q[2] : R.q[3]);
  const float l1 = __fmul_rn(__ll2float_rn(e[1]), inv);
  const float l2 = __fmul_rn(__ll2float_rn(e[2]), inv);
  const float key = __fadd_rn(qa, __fadd_rn(__fmul_rn(l1, __fsub_rn(qb, qa)), __fmul_rn(l2, __fsub_rn(qc, qa))));
  const uint32_t jl = (uint32_t)(rec - V.quad_base);
  sk = ((unsigned long long)__float_as_uint(key) << 32) | (2u * jl + (uint32_t)t);
  if (col) {
    if (V.color_mode == LR_COLOR_FLAT) {
      *col = __ldg(reinterpret_cast<const float4*>(V.col) + jl);
    } else {
      // perspective-correct: sum_k (l_k q_k) c_k / sum_k l_k q_k
      uint4 q4;
      if (V.idx) q4 = __ldg(reinterpret_cast<const uint4*>(V.idx) + jl);
      else q4 = make_uint4(4 * jl, 4 * jl + 1, 4 * jl + 2, 4 * jl + 3);
      const uint32_t va = q4.x;
      const uint32_t vb = ib == 1 ? q4.y : (ib == 2 ? q4.z : q4.w);
      const uint32_t vc = ic == 1 ? q4.y : (ic == 2 ? q4.z : q4.w);
      const float wa = __fmul_rn(__ll2float_rn(e[0]), inv) * qa, wb = l1 * qb, wc = l2 * qc;
      // lit views: 32 bytes per vertex, the colour then the normal
      const bool lit = V.color_mode == LR_COLOR_LIT;
      const int stride = lit ? 2 : 1;
      const float4* cv = reinterpret_cast<const float4*>(V.col);
      const float4 ca = __ldg(cv + (size_t)stride * va);
      const float4 cb = __ldg(cv + (size_t)stride * vb);
      const float4 cc = __ldg(cv + (size_t)stride * vc);
      const float r = 1.0f / (wa + wb + wc);
      *col = make_float4((wa * ca.x + wb * cb.x + wc * cc.x) * r, (wa * ca.y + wb * cb.y + wc * cc.y) * r,
                         (wa * ca.z + wb * cb.z + wc * cc.z) * r, (wa * ca.w + wb * cb.w + wc * cc.w) * r);
      if (lit) {
        // two-sided Lambert term of the interpolated normal's direction, plus ambient
        const float4 na = __ldg(cv + 2ull * va + 1), nb = __ldg(cv + 2ull * vb + 1), nc = __ldg(cv + 2ull * vc + 1);
        const float nx = wa * na.x + wb * nb.x + wc * nc.x;
        const float ny = wa * na.y + wb * nb.y + wc * nc.y;
        const float nz = wa * na.z + wb * nb.z + wc * nc.z;
        const float nn = nx * nx + ny * ny + nz * nz;
        const float d = fabsf(nx * V.light[0] + ny * V.light[1] + nz * V.light[2]);
        const float lam = nn > 0.f ? fminf(d * rsqrtf(nn), 1.0f) : 0.f;
        const float f = V.light[3] + (1.0f - V.light[3]) * lam;
        col->x *= f;
        col->y *= f;
        col->z *= f;
      }
    }
  }
  return true;
}

__device__ __forceinline__ bool frag_eval(const Ws& ws, const ViewDev& V, uint32_t rec, int t, int px, int py,
                                          unsigned long long& sk, float4* col) {
  const QuadRec R = load_rec(ws.rec, rec);
  return frag_eval_r(ws, V, R, rec, t, px, py, sk, col);
}

// descending bitonic sort of buf[0, n2) by one warp (n2 a power of two >= 32)
static __device__ void warp_sort_desc(unsigned long long* buf, int n2) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < (n2 >> 1); i += 32) {
        const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
        const int hi = lo | j;
        const bool down = (lo & k) == 0;
        const unsigned long long a = buf[lo], b = buf[hi];
        if ((a < b) == down) { buf[lo] = b; buf[hi] = a; }
      }
      __syncwarp();
    }
  }
}

__device__ __forceinline__ int pow2_at_least(int n) {
  int p = 32;
  while (p < n) p <<= 1;
  return p;
}

// Front-to-back composite of the sorted fragments buf[0, m) of pixel (px, py) onto the
// running (cr, cg, cb, T): each lane composites a contiguous segment, then an inclusive
// scan of (C, T) pairs with (C1, T1) o (C2, T2) = (C1 + T1 C2, T1 T2) combines them in
// order. With grad, also accumulates the per-quad RGBA gradient (flat colours): each lane
// walks its segment again from the exact prefix of the lanes before it.
static __device__ void composite_sorted(const Ws& ws, const ViewDev& V, const unsigned long long* buf, int m, int px,
                                 int py, float& cr, float& cg, float& cb, float& T, const GradPixel* gp) {
  const int lane = threadIdx.x & 31;
  if (ws.t_min > 0.0f) {
    // alpha threshold (forward only): whether a fragment is blended depends on the exact
    // running product T, which the segmented scan below rounds differently, so one lane
    // walks the fragments in order with the rasteriser's blend and stops where T <= t_min
    if (lane == 0) {
      for (int k = 0; k < m && T > ws.t_min; ++k) {
        const uint32_t id = (uint32_t)buf[k];
        float4 col;
        unsigned long long dummy;
        frag_eval(ws, V, (uint32_t)(V.quad_base + (id >> 1)), (int)(id & 1u), px, py, dummy, &col);
        const float w = T * col.w;
        cr += w * col.x; cg += w * col.y; cb += w * col.z;
        T *= 1.0f - col.w;
      }
    }
    cr = __shfl_sync(0xffffffffu, cr, 0); cg = __shfl_sync(0xffffffffu, cg, 0);
    cb = __shfl_sync(0xffffffffu, cb, 0); T = __shfl_sync(0xffffffffu, T, 0);
    return;
  }
  const int seg = (m + 31) / 32;
  float sr = 0.f, sg = 0.f, sb = 0.f, sT = 1.f;
  for (int k = lane * seg; k < min(m, (lane + 1) * seg); ++k) {
    const unsigned long long sk = buf[k];
    const uint32_t id = (uint32_t)sk;
    float4 col;
    unsigned long long dummy;
    frag_eval(ws, V, (uint32_t)(V.quad_base + (id >> 1)), (int)(id & 1u), px, py, dummy, &col);
    const float w = sT * col.w;
    sr += w * col.x; sg += w * col.y; sb += w * col.z;
    sT *= 1.0f - col.w;
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float pr = __shfl_up_sync(0xffffffffu, sr, o), pg = __shfl_up_sync(0xffffffffu, sg, o);
    const float pb = __shfl_up_sync(0xffffffffu, sb, o), pT = __shfl_up_sync(0xffffffffu, sT, o);
    if (lane >= o) {
      sr = pr + pT * sr; sg = pg + pT * sg; sb = pb + pT * sb; sT = pT * sT;
    }
  }
  if (gp) {
    float er = __shfl_up_sync(0xffffffffu, sr, 1), eg = __shfl_up_sync(0xffffffffu, sg, 1);
    float eb = __shfl_up_sync(0xffffffffu, sb, 1), eT = __shfl_up_sync(0xffffffffu, sT, 1);
    if (lane == 0) { er = eg = eb = 0.f; eT = 1.f; }
    float wr = cr + T * er, wg = cg + T * eg, wb = cb + T * eb, wT = T * eT;
    for (int k = lane * seg; k < min(m, (lane + 1) * seg); ++k) {
      const uint32_t id = (uint32_t)buf[k];
      const uint32_t j = id >> 1;
      const float4 col = __ldg(reinterpret_cast<const float4*>(V.col) + j);
      const float w = wT * col.w;
      wr += w * col.x; wg += w * col.y; wb += w * col.z;
      const float om = 1.0f - col.w;
      float da = gp->gr * wT * col.x + gp->gg * wT * col.y + gp->gb * wT * col.z;
      if (om > 1e-6f) {
        const float inv = 1.0f / om;
        da -= (gp->gr * (gp->fr - wr) + gp->gg * (gp->fg - wg) + gp->gb * (gp->fb - wb)) * inv;
        da += gp->ga * gp->fT * inv;
      }
      float* gq = gp->grad + 4ull * j;
      atomicAdd(gq + 0, gp->gr * w);
      atomicAdd(gq + 1, gp->gg * w);
      atomicAdd(gq + 2, gp->gb * w);
      atomicAdd(gq + 3, da);
      wT *= om;
    }
  }
  sr = __shfl_sync(0xffffffffu, sr, 31); sg = __shfl_sync(0xffffffffu, sg, 31);
  sb = __shfl_sync(0xffffffffu, sb, 31); sT = __shfl_sync(0xffffffffu, sT, 31);
  cr += T * sr; cg += T * sg; cb += T * sb; T *= sT;
}

// The exact path for one pixel (flattened id pid) by one warp, with buf a BUF-entry
// shared-memory buffer (BUF a power of two >= 64; a pass composites the KEEP = 15/32 BUF
// nearest remaining fragments). BWD: instead of writing the pixel, accumulate the gradient
// of the flat per-quad RGBA (same formulas as the rasteriser's backward).
template <bool BWD, int BUF>
__device__ void overflow_pixel(const Ws& ws, long long pid, unsigned long long* buf) {
  constexpr int KEEP = BUF * 15 / 32;
  const int lane = threadIdx.x & 31;
  const int v = view_of_pixel(ws.views, ws.n_views, pid);
  const ViewDev& V = ws.views[v];
  const long long pidx = pid - V.pix_base;
  const int px = (int)(pidx % V.width), py = (int)(pidx / V.width);
  const int lg = ws.bin_log2, B = 1 << lg;
  const int bin_g = V.bin_base + (py >> lg) * V.nbx + (px >> lg);
  const int hb = ((py & (B - 1)) / kHbH) * bin_hb_cols(lg) + (px & (B - 1)) / kHbW;
  const uint32_t off = ws.bin_off[bin_g];
  const int n = (int)(ws.bin_off[bin_g + 1] - off);

  float cr = 0.f, cg = 0.f, cb = 0.f, T = 1.f;
  unsigned long long tau = kSent;   // exclusive upper bound of the fragments still to do
  GradPixel gp;
  if (BWD) {
    const float4 gq = reinterpret_cast<const float4*>(ws.grad_out)[pidx];
    const float4 fq = reinterpret_cast<const float4*>(ws.fwd)[pidx];
    gp.gr = gq.x; gp.gg = gq.y; gp.gb = gq.z; gp.ga = gq.w;
    gp.fr = fq.x; gp.fg = fq.y; gp.fb = fq.z; gp.fT = 1.0f - fq.w;
    gp.grad = ws.grad_col;
  }
  for (;;) {
    int nbuf = 0, below = 0;
    unsigned long long lb = 0;     // exclusive lower bound once the buffer was cut back
    const uint32_t* row = hb_row(ws, off, bin_g, n, hb);
    const int nw = (n + 31) >> 5;
    for (int g = 0; g < nw; g += 32) {
      BitRounds br;
      br.prepare(g + lane < nw ? __ldg(row + g + lane) : 0u, lane);
      // candidates of the pixel's half-block, 32 per round; the next round's reference and
      // quad record are loaded while the current round is evaluated
      int jn = br.get(0, lane);
      uint32_t recn = jn >= 0 ? ~(uint32_t)ws.refs[off + 32 * g + jn] : 0u;
      QuadRec Rn = {};
      if (jn >= 0) Rn = load_rec(ws.rec, recn);
      for (int r0 = 0; r0 < br.total; r0 += 32) {
        const int j = jn;
        const uint32_t rec = recn;
        const QuadRec R = Rn;
        if (r0 + 32 < br.total) {
          jn = br.get(r0 + 32, lane);
          recn = jn >= 0 ? ~(uint32_t)ws.refs[off + 32 * g + jn] : 0u;
          if (jn >= 0) Rn = load_rec(ws.rec, recn);
        }
        // the exact test below decides coverage
        const bool hit = j >= 0;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          unsigned long long sk = 0;
          const bool cov = hit && frag_eval_r(ws, V, R, rec, t, px, py, sk, nullptr) && sk < tau;
          below += __popc(__ballot_sync(0xffffffffu, cov));
          const bool keep = cov && sk > lb;
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          if (keep) buf[nbuf + __popc(m & ((1u << lane) - 1u))] = sk;
          nbuf += __popc(m);
          __syncwarp();
          if (nbuf >= BUF - 32) {
            const int n2 = pow2_at_least(nbuf);
            for (int k = nbuf + lane; k < n2; k += 32) buf[k] = 0ull;
            __syncwarp();
            warp_sort_desc(buf, n2);
            nbuf = KEEP;
            lb = buf[KEEP - 1];
          }
        }
      }
    }
    const int n2 = pow2_at_least(nbuf);
    for (int k = nbuf + lane; k < n2; k += 32) buf[k] = 0ull;
    __syncwarp();
    warp_sort_desc(buf, n2);
    const int m = min(nbuf, KEEP);
    composite_sorted(ws, V, buf, m, px, py, cr, cg, cb, T, BWD ? &gp : nullptr);
    if (below <= KEEP || m == 0) break;
    if (!BWD && ws.t_min > 0.0f && !(T > ws.t_min)) break;   // alpha threshold reached
    tau = buf[m - 1];
    __syncwarp();
  }
  if (!BWD && lane == 0) write_pixel(V, pidx, cr, cg, cb, T);
  __syncwarp();
}

}  // namespace lr
