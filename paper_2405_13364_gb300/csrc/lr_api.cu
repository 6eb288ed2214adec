// lr_api.cu -- the C ABI (include/lr.h): argument checking, workspace layout, and the
// launch sequence of one render:
//
//   k_init         zero control block and bin counters; view descriptors -> workspace
//                  (kernel parameters, no host buffer; k_write_views for views past 16)
//   k_setup        Stage 1  (Sec. 2, "Stage 1: quad setup")
//   k_bin_count    Stage 2, Phase 1
//   k_bin_scan     Stage 2, Phase 2
//   k_bin_scatter  Stage 2, Phase 3
//   k_bin_sort     Stage 3, Phase 2's depth sort of each bin's references (stage 1 of 2)
//   k_raster       Stage 3: coverage, per-pixel sorter (stage 2 of 2), blending
//   k_overflow     exact full sort of the pixels the sorter flagged
//
// Every grid size depends only on host-known sizes (quads, bins, SM count); all
// data-dependent sizes are read on the device, so the sequence has no host round trip
// and can be captured into a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lr_common.cuh"
#include "lr_raster.cuh"
#include "lr_serve.h"

namespace lr {
__global__ void k_init(Ws ws, unsigned long long refs_cap, ViewChunk views, ViewDev* views_dst);
__global__ void k_setup(Ws ws);
__global__ void k_bin_count(Ws ws);
__global__ void k_bin_scan(Ws ws);
__global__ void k_bin_scatter(Ws ws);
__global__ void k_bin_sort(Ws ws);
__global__ void k_bin_sort_big(Ws ws);
cudaError_t overflow_occupancy(int* blocks_per_sm);
cudaError_t launch_overflow(bool bwd, const Ws& ws, int grid, cudaStream_t st, bool pdl);

#define LR_DECLARE_RASTER(KK)                                                                     \
  cudaError_t prepare_raster_##KK(int* blocks_flat, int* blocks_vtx, int* blocks_bwd, int* blocks_lit); \
  cudaError_t launch_raster_##KK(int mode, const Ws& ws, int grid, cudaStream_t st);
LR_DECLARE_RASTER(1)
LR_DECLARE_RASTER(2)
LR_DECLARE_RASTER(3)
LR_DECLARE_RASTER(4)
LR_DECLARE_RASTER(6)
LR_DECLARE_RASTER(8)
LR_DECLARE_RASTER(12)
#define LR_DECLARE_RASTER8(KK)                                                                    \
  cudaError_t prepare_raster8_##KK(int* blocks_flat, int* blocks_vtx);                            \
  cudaError_t launch_raster8_##KK(int mode, const Ws& ws, int grid, cudaStream_t st);
LR_DECLARE_RASTER8(1)
LR_DECLARE_RASTER8(2)
LR_DECLARE_RASTER8(3)
#define LR_DECLARE_RASTER_STRIP(KK)                                                               \
  cudaError_t prepare_raster_strip_##KK(int* blocks_flat, int* blocks_vtx);                       \
  cudaError_t launch_raster_strip_##KK(int mode, const Ws& ws, int grid, cudaStream_t st);
LR_DECLARE_RASTER_STRIP(1)
LR_DECLARE_RASTER_STRIP(2)
LR_DECLARE_RASTER_STRIP(3)

__global__ void k_write_views(ViewChunk chunk, ViewDev* dst) {
  pdl_begin();
  const int i = threadIdx.x;
  if (i < chunk.count) dst[chunk.first + i] = chunk.v[i];
}

typedef cudaError_t (*PrepareFn)(int*, int*, int*, int*);
typedef cudaError_t (*LaunchFn)(int, const Ws&, int, cudaStream_t);   // mode 0 flat, 1 colours, 2 backward
typedef cudaError_t (*Prepare8Fn)(int*, int*);

// A sorter capacity's rasterisers: 8x4 half-blocks (every mode) and, for K <= 3, 8x8 blocks
// (forward exact renders, flat or carried colours, with or without the coverage hash).
struct RasterVariant {
  int k;
  PrepareFn prepare;
  LaunchFn launch;
  Prepare8Fn prepare8;
  LaunchFn launch8;
  Prepare8Fn prepare_strip;   // the per-strip shared set-up (lr_raster_strip.cuh)
  LaunchFn launch_strip;
};

static const RasterVariant kVariants[] = {
    {1, prepare_raster_1, launch_raster_1, prepare_raster8_1, launch_raster8_1, prepare_raster_strip_1, launch_raster_strip_1},
    {2, prepare_raster_2, launch_raster_2, prepare_raster8_2, launch_raster8_2, prepare_raster_strip_2, launch_raster_strip_2},
    {3, prepare_raster_3, launch_raster_3, prepare_raster8_3, launch_raster8_3, prepare_raster_strip_3, launch_raster_strip_3},
    {4, prepare_raster_4, launch_raster_4, nullptr, nullptr, nullptr, nullptr},
    {6, prepare_raster_6, launch_raster_6, nullptr, nullptr, nullptr, nullptr},
    {8, prepare_raster_8, launch_raster_8, nullptr, nullptr, nullptr, nullptr},
    {12, prepare_raster_12, launch_raster_12, nullptr, nullptr, nullptr, nullptr},
};

struct Layout {
  int bin_log2 = kBinLog2Default;
  size_t ctrl, views, rec, rec_rect, rec_info, rec_rep, bin_count, bin_off, bin_cursor, bin_order, chunk_span;
  size_t refs, refs_tmp, ref_hb, ovf_list, total;
  long long total_quads = 0, total_pix = 0, refs_cap = 0;
  int total_bins = 0, total_chunks = 0;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout. The two bin-reference arrays come last; their capacity is whatever the
// workspace holds beyond the fixed part (set_capacity), so a caller that hit
// LR_ERR_OVERFLOW can pass a larger workspace without recreating the context.
static Layout make_layout(int n, const long long* Q, const int* W, const int* H, int lg) {
  Layout L;
  L.bin_log2 = lg;
  const int B = 1 << lg;
  for (int i = 0; i < n; ++i) {
    const int nbx = (W[i] + B - 1) / B, nby = (H[i] + B - 1) / B;
    L.total_quads += Q[i];
    L.total_pix += (long long)W[i] * H[i];
    L.total_bins += nbx * nby;
    L.total_chunks += (int)((Q[i] + kChunkQuads - 1) / kChunkQuads);
  }
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
  L.ctrl = take(sizeof(Ctrl));
  L.views = take(sizeof(ViewDev) * (size_t)n);
  L.rec = take(sizeof(int4) * 4 * (size_t)L.total_quads);
  L.rec_rect = take(sizeof(uint2) * (size_t)L.total_quads);
  L.rec_info = take(sizeof(uint32_t) * (size_t)L.total_quads);
  L.rec_rep = take(sizeof(float) * (size_t)L.total_quads);
  L.bin_count = take(sizeof(uint32_t) * (size_t)L.total_bins);
  L.bin_off = take(sizeof(uint32_t) * ((size_t)L.total_bins + 1));
  L.bin_cursor = take(sizeof(uint32_t) * (size_t)L.total_bins);
  L.chunk_span = take(sizeof(uint2) * (size_t)L.total_chunks);
  L.bin_order = take(sizeof(uint32_t) * (size_t)L.total_bins);
  L.ovf_list = take(sizeof(uint32_t) * (size_t)L.total_pix);
  L.refs = o;      // refs and refs_tmp follow; see set_capacity
  L.total = o;
  return L;
}

static const long long kMaxRefs = 0xFFFFFF00LL;   // offsets are 32-bit

static long long default_refs(const Layout& L, int ref_factor) {
  return std::min((long long)ref_factor * L.total_quads + 64LL * L.total_bins + 1024, kMaxRefs);
}

// per reference: the sort key, its merge buffer slot and its mw words of the half-block
// bitmap (plus up to mrows padding words per bin)
static size_t bytes_for_refs(const Layout& L, long long refs) {
  const size_t mw = (size_t)bin_mw(L.bin_log2), mrows = (size_t)bin_mrows(L.bin_log2);
  return L.refs + align256(sizeof(unsigned long long) * (size_t)refs) * 2 +
         align256(sizeof(uint32_t) * (mw * (size_t)refs + mrows * (size_t)L.total_bins));
}

// capacity from the bytes available, placing refs_tmp and ref_hb after refs
static void set_capacity(Layout& L, size_t ws_bytes) {
  long long cap = 0;
  const size_t mw = (size_t)bin_mw(L.bin_log2), mrows = (size_t)bin_mrows(L.bin_log2);
  const size_t fixed = L.refs + mrows * sizeof(uint32_t) * (size_t)L.total_bins + 1024;
  if (ws_bytes > fixed) cap = (long long)((ws_bytes - fixed) / (2 * sizeof(unsigned long long) + mw * sizeof(uint32_t)));
  cap = std::min(cap, kMaxRefs);
  cap &= ~63LL;
  while (cap > 0 && bytes_for_refs(L, cap) > ws_bytes) cap -= 64;
  L.refs_cap = std::max(cap, 0LL);
  L.refs_tmp = L.refs + align256(sizeof(unsigned long long) * (size_t)L.refs_cap);
  L.ref_hb = L.refs_tmp + align256(sizeof(unsigned long long) * (size_t)L.refs_cap);
  L.total = bytes_for_refs(L, L.refs_cap);
}

static Ws make_ws(const Layout& L, void* base, int n_views) {
  char* b = static_cast<char*>(base);
  Ws w;
  memset(&w, 0, sizeof(w));
  w.ctrl = reinterpret_cast<Ctrl*>(b + L.ctrl);
  w.views = reinterpret_cast<const ViewDev*>(b + L.views);
  w.n_views = n_views;
  w.total_bins = L.total_bins;
  w.total_quads = L.total_quads;
  w.total_pix = L.total_pix;
  w.refs_cap = L.refs_cap;
  w.bin_log2 = L.bin_log2;
  w.rec = reinterpret_cast<int4*>(b + L.rec);
  w.rec_rect = reinterpret_cast<uint2*>(b + L.rec_rect);
  w.rec_info = reinterpret_cast<uint32_t*>(b + L.rec_info);
  w.rec_rep = reinterpret_cast<float*>(b + L.rec_rep);
  w.bin_count = reinterpret_cast<uint32_t*>(b + L.bin_count);
  w.bin_off = reinterpret_cast<uint32_t*>(b + L.bin_off);
  w.bin_cursor = reinterpret_cast<uint32_t*>(b + L.bin_cursor);
  w.chunk_span = reinterpret_cast<uint2*>(b + L.chunk_span);
  w.bin_order = reinterpret_cast<uint32_t*>(b + L.bin_order);
  w.refs = reinterpret_cast<unsigned long long*>(b + L.refs);
  w.refs_tmp = reinterpret_cast<unsigned long long*>(b + L.refs_tmp);
  w.ref_hb = reinterpret_cast<uint32_t*>(b + L.ref_hb);
  w.ovf_list = reinterpret_cast<uint32_t*>(b + L.ovf_list);
  return w;
}

}  // namespace lr

using namespace lr;

// A rasteriser variant (sorter capacity K) with its resident CTAs per SM for each colour
// layout, the launch grid of its persistent kernels.
struct VariantState {
  const RasterVariant* v = nullptr;
  int flat = 1, vtx = 1, bwd = 1, lit = 1;
  int flat8 = 1, vtx8 = 1;     // the 8x8-block kernels (when the capacity has them)
  int flat_s = 1, vtx_s = 1;   // the strip kernels
};

struct lr_ctx {
  int device = 0;
  int sms = 0;
  lr_config cfg;
  VariantState vs[sizeof(kVariants) / sizeof(kVariants[0])];
  int variant = 0;             // index of the context's default sorter capacity in vs
  int pdl_override = -1;       // -1: as cfg.flags say; 0 / 1: this render without / with PDL
  int bin_log2 = kBinLog2Default;   // from cfg.bin_size
  float light[4] = {0.f, 0.f, 1.f, 0.25f};   // LR_COLOR_LIT: unit direction toward the light, ambient
  int ovf_blocks = 1;
  // last render, for lr_get_stats
  cudaStream_t last_stream = nullptr;
  void* last_ws = nullptr;
  int last_views = 0;
  long long last_quads = 0;
  long long last_cap = 0;
  bool have_last = false;
  bool last_timed = false;
  cudaEvent_t ev[9] = {};
  Ctrl* host_ctrl = nullptr;   // pinned
  lr_server* server = nullptr;
  char err[512] = {0};
};

lr_server** lr_internal_server_slot(lr_ctx* ctx) { return &ctx->server; }
void lr_internal_set_pdl(lr_ctx* ctx, int pdl) { ctx->pdl_override = pdl; }
const lr_config* lr_internal_config(const lr_ctx* ctx) { return &ctx->cfg; }

static lr_status fail(lr_ctx* c, lr_status s, const char* fmt, const char* detail = "") {
  if (c) snprintf(c->err, sizeof(c->err), fmt, detail);
  return s;
}

static lr_status cuda_fail(lr_ctx* c, cudaError_t e, const char* what) {
  if (c) snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LR_ERR_OOM : LR_ERR_CUDA;
}

extern "C" lr_status lr_create(const lr_config* config, lr_ctx** out_ctx) {
  if (!out_ctx) return LR_ERR_INVALID_ARG;
  *out_ctx = nullptr;
  lr_ctx* c = new (std::nothrow) lr_ctx();
  if (!c) return LR_ERR_OOM;
  memset(&c->cfg, 0, sizeof(c->cfg));
  if (config) c->cfg = *config;
  lr_config& g = c->cfg;
  if (g.max_width <= 0) g.max_width = 2560;
  if (g.max_height <= 0) g.max_height = 2048;
  if (g.sorter_k <= 0) g.sorter_k = 3;
  if (g.ref_factor <= 0) g.ref_factor = 4;
  if (g.bin_size <= 0) g.bin_size = 1 << kBinLog2Default;
  if (g.block_h <= 0) g.block_h = kHbH;
  c->bin_log2 = g.bin_size == 16 ? 4 : (g.bin_size == 32 ? 5 : (g.bin_size == 64 ? 6 : -1));
  if (g.max_width > 65535 || g.max_height > 65535 || g.raster_ctas_per_sm < 0 || c->bin_log2 < 0 ||
      (g.block_h != 4 && g.block_h != 8) || g.shared_setup < 0 || g.shared_setup > 1) {
    delete c;
    return LR_ERR_INVALID_ARG;
  }
  c->variant = -1;
  for (int i = 0; i < (int)(sizeof(kVariants) / sizeof(kVariants[0])); ++i)
    if (kVariants[i].k == g.sorter_k) c->variant = i;
  if (c->variant < 0) {
    delete c;
    return LR_ERR_INVALID_ARG;
  }
  cudaError_t e;
  if (g.device > 0) {
    e = cudaSetDevice(g.device);
    if (e != cudaSuccess) { delete c; return LR_ERR_CUDA; }
  }
  e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  // every sorter capacity is prepared, so that a view may ask for its own (lr_view.sorter_k)
  for (int i = 0; i < (int)(sizeof(kVariants) / sizeof(kVariants[0])) && e == cudaSuccess; ++i) {
    VariantState& V = c->vs[i];
    V.v = &kVariants[i];
    e = V.v->prepare(&V.flat, &V.vtx, &V.bwd, &V.lit);
    if (e == cudaSuccess && V.v->prepare8 && g.block_h == 8) e = V.v->prepare8(&V.flat8, &V.vtx8);
    if (e == cudaSuccess && V.v->prepare_strip && g.shared_setup) e = V.v->prepare_strip(&V.flat_s, &V.vtx_s);
    int* all[] = {&V.flat, &V.vtx, &V.bwd, &V.lit, &V.flat8, &V.vtx8, &V.flat_s, &V.vtx_s};
    for (int* x : all) {
      if (g.raster_ctas_per_sm > 0) *x = std::min(*x, g.raster_ctas_per_sm);
      *x = std::max(*x, 1);
    }
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bin_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSortSmemBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bin_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSortBigSmemBytes);
  if (e == cudaSuccess) e = overflow_occupancy(&c->ovf_blocks);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c->host_ctrl), sizeof(Ctrl));
  for (int i = 0; i < 9 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
  if (e != cudaSuccess) {
    lr_status s = e == cudaErrorMemoryAllocation ? LR_ERR_OOM : LR_ERR_CUDA;
    lr_destroy(c);
    return s;
  }
  c->ovf_blocks = std::max(c->ovf_blocks, 1);
  *out_ctx = c;
  return LR_OK;
}

extern "C" lr_status lr_set_lighting(lr_ctx* ctx, const float* light_dir, float ambient) {
  if (!ctx || !light_dir) return LR_ERR_INVALID_ARG;
  const double x = light_dir[0], y = light_dir[1], z = light_dir[2];
  const double n = std::sqrt(x * x + y * y + z * z);
  if (!(n > 0.0) || !std::isfinite(n)) return fail(ctx, LR_ERR_INVALID_ARG, "light direction must be finite and non-zero%s");
  if (!(ambient >= 0.0f && ambient <= 1.0f)) return fail(ctx, LR_ERR_INVALID_ARG, "ambient must lie in [0, 1]%s");
  ctx->light[0] = (float)(x / n);
  ctx->light[1] = (float)(y / n);
  ctx->light[2] = (float)(z / n);
  ctx->light[3] = ambient;
  return LR_OK;
}

const float* lr_internal_light(const lr_ctx* ctx) { return ctx->light; }

extern "C" lr_status lr_destroy(lr_ctx* ctx) {
  if (!ctx) return LR_ERR_INVALID_ARG;
  if (ctx->server) lr_server_stop(ctx);
  for (int i = 0; i < 9; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  if (ctx->host_ctrl) cudaFreeHost(ctx->host_ctrl);
  delete ctx;
  return LR_OK;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static lr_status check_view(lr_ctx* c, const lr_view& v) {
  if (v.width <= 0 || v.height <= 0) return fail(c, LR_ERR_INVALID_ARG, "width and height must be positive%s");
  if (v.width > c->cfg.max_width || v.height > c->cfg.max_height)
    return fail(c, LR_ERR_TOO_LARGE, "resolution above the context maximum%s");
  const lr_quads& q = v.quads;
  if (q.num_quads < 0 || q.num_vertices < 0) return fail(c, LR_ERR_INVALID_ARG, "negative sizes%s");
  if (q.num_quads > 0x7FFFFFFFLL / 2) return fail(c, LR_ERR_TOO_LARGE, "too many quads%s");
  if (q.num_quads > 0) {
    if (!q.positions || !q.colors) return fail(c, LR_ERR_INVALID_ARG, "null positions or colors%s");
    if (!aligned(q.positions, 16) || !aligned(q.colors, 16) || (q.indices && !aligned(q.indices, 16)))
      return fail(c, LR_ERR_INVALID_ARG, "positions, colors and indices must be 16-byte aligned%s");
    if (q.color_mode != LR_COLOR_FLAT && q.color_mode != LR_COLOR_VERTEX && q.color_mode != LR_COLOR_LIT)
      return fail(c, LR_ERR_INVALID_ARG, "unknown color_mode%s");
  }
  if (!v.target.rgba || !aligned(v.target.rgba, 16)) return fail(c, LR_ERR_INVALID_ARG, "rgba output must be non-null and 16-byte aligned%s");
  if ((v.target.rgba8 && !aligned(v.target.rgba8, 4)) || (v.target.frag_count && !aligned(v.target.frag_count, 4)) ||
      (v.target.cov_hash && !aligned(v.target.cov_hash, 8)) || (v.target.exact_mask && !aligned(v.target.exact_mask, 4)) ||
      (v.owned_tiles && !aligned(v.owned_tiles, 4)))
    return fail(c, LR_ERR_INVALID_ARG, "misaligned optional output%s");
  const float n = v.camera.near_z, f = v.camera.far_z;
  if (!(n > 0.0f) || !(f >= n) || !(f < 3.4e38f)) return fail(c, LR_ERR_INVALID_ARG, "need 0 < near <= far < inf%s");
  if (v.sorter_k) {
    bool known = false;
    for (const auto& kv : kVariants) known |= kv.k == v.sorter_k;
    if (!known) return fail(c, LR_ERR_INVALID_ARG, "sorter_k must be 0 or one of 1, 2, 3, 4, 6, 8, 12%s");
  }
  return LR_OK;
}

lr_status lr_internal_check_view(lr_ctx* ctx, const lr_view* view) { return check_view(ctx, *view); }

static lr_status layout_for(lr_ctx* c, int n, const lr_view* views, Layout* out) {
  std::vector<long long> Q(n);
  std::vector<int> W(n), H(n);
  long long total_pix = 0;
  for (int i = 0; i < n; ++i) {
    Q[i] = views[i].quads.num_quads;
    W[i] = views[i].width;
    H[i] = views[i].height;
    total_pix += (long long)W[i] * H[i];
  }
  *out = make_layout(n, Q.data(), W.data(), H.data(), c->bin_log2);
  if (out->total_quads > 0x7FFFFFFFLL || total_pix > 0xFFFFFFFFLL)
    return fail(c, LR_ERR_TOO_LARGE, "batch too large%s");
  return LR_OK;
}

extern "C" lr_status lr_workspace_size(const lr_ctx* ctx, int64_t num_quads, int32_t width, int32_t height,
                                       size_t* out_bytes) {
  if (!ctx || !out_bytes || num_quads < 0 || width <= 0 || height <= 0) return LR_ERR_INVALID_ARG;
  if (width > ctx->cfg.max_width || height > ctx->cfg.max_height) return LR_ERR_TOO_LARGE;
  const long long q = num_quads;
  const int w = width, h = height;
  Layout L = make_layout(1, &q, &w, &h, ctx->bin_log2);
  *out_bytes = bytes_for_refs(L, default_refs(L, ctx->cfg.ref_factor));
  return LR_OK;
}

extern "C" lr_status lr_workspace_size_batch(const lr_ctx* ctx, int32_t n_views, const lr_view* views,
                                             size_t* out_bytes) {
  return lr_workspace_size_refs(ctx, n_views, views, -1, out_bytes);
}

extern "C" lr_status lr_workspace_size_refs(const lr_ctx* ctx, int32_t n_views, const lr_view* views,
                                            int64_t bin_refs, size_t* out_bytes) {
  if (!ctx || !views || n_views <= 0 || !out_bytes) return LR_ERR_INVALID_ARG;
  Layout L;
  lr_status s = layout_for(const_cast<lr_ctx*>(ctx), n_views, views, &L);
  if (s != LR_OK) return s;
  if (bin_refs > kMaxRefs) return LR_ERR_TOO_LARGE;
  const long long refs = bin_refs < 0 ? default_refs(L, ctx->cfg.ref_factor) : (long long)bin_refs;
  *out_bytes = bytes_for_refs(L, refs);
  return LR_OK;
}

extern "C" lr_status lr_workspace_layout(const lr_ctx* ctx, int32_t n_views, const lr_view* views,
                                         size_t workspace_bytes, lr_ws_layout* out) {
  if (!ctx || !views || n_views <= 0 || !out) return LR_ERR_INVALID_ARG;
  Layout L;
  lr_status s = layout_for(const_cast<lr_ctx*>(ctx), n_views, views, &L);
  if (s != LR_OK) return s;
  set_capacity(L, workspace_bytes);
  out->rec = L.rec;
  out->rec_rect = L.rec_rect;
  out->rec_info = L.rec_info;
  out->bin_count = L.bin_count;
  out->bin_off = L.bin_off;
  out->refs = L.refs;
  out->total_quads = L.total_quads;
  out->total_bins = L.total_bins;
  out->refs_capacity = L.refs_cap;
  return LR_OK;
}

static inline void rec(lr_ctx* c, bool timed, int i, cudaStream_t s) {
  if (timed) cudaEventRecord(c->ev[i], s);
}

struct BwdArgs {
  const float* fwd;
  const float* grad_out;
  float* grad_colors;
  const uint32_t* exact_mask;
};

// A render, checked and laid out on the host: workspace pointers and view descriptors.
struct Prepared {
  Layout L;
  std::vector<ViewDev> vd;
  bool any_vertex = false;
  bool any_hash = false;   // a view asks for the coverage hash (selects the hashing rasteriser)
  bool any_lit = false;    // a view has lit colours (selects the shading rasteriser)
  Ws ws;
  ViewDev* views_dev = nullptr;
  int variant = 0;         // the batch's sorter capacity (index into lr_ctx::vs)
};

static void describe_views(int32_t n_views, const lr_view* views, std::vector<ViewDev>& vd, bool* any_vertex,
                           bool* any_hash, bool* any_lit, const float* light, int lg) {
  const int B = 1 << lg;
  vd.resize(n_views);
  long long qb = 0, pb = 0;
  int bb = 0, cb = 0;
  *any_vertex = false;
  *any_hash = false;
  *any_lit = false;
  for (int i = 0; i < n_views; ++i) {
    const lr_view& v = views[i];
    ViewDev& d = vd[i];
    memset(&d, 0, sizeof(d));
    d.pos = v.quads.positions;
    d.idx = v.quads.indices;
    d.col = v.quads.colors;
    d.out = v.target.rgba;
    d.out8 = v.target.rgba8;
    d.cnt = v.target.frag_count;
    d.hash = reinterpret_cast<unsigned long long*>(v.target.cov_hash);
    d.xmask = v.target.exact_mask;
    d.owned = v.owned_tiles;
    const float* M = v.camera.view_proj;
    for (int k = 0; k < 4; ++k) {
      d.m[k] = M[k];
      d.m[4 + k] = M[4 + k];
      d.m[8 + k] = M[12 + k];
    }
    for (int k = 0; k < 4; ++k) d.light[k] = light[k];
    d.near_z = v.camera.near_z;
    d.far_z = v.camera.far_z;
    d.half_w = 0.5f * (float)v.width;
    d.half_h = 0.5f * (float)v.height;
    d.num_vertices = v.quads.num_vertices;
    d.num_quads = (int)v.quads.num_quads;
    d.color_mode = v.quads.color_mode;
    d.width = v.width;
    d.height = v.height;
    d.nbx = (v.width + B - 1) / B;
    d.nby = (v.height + B - 1) / B;
    d.quad_base = qb;
    d.pix_base = pb;
    d.bin_base = bb;
    d.chunk_base = cb;
    qb += v.quads.num_quads;
    pb += (long long)v.width * v.height;
    bb += d.nbx * d.nby;
    cb += (int)((v.quads.num_quads + kChunkQuads - 1) / kChunkQuads);
    *any_vertex |= (v.quads.color_mode == LR_COLOR_VERTEX && v.quads.num_quads > 0);
    *any_hash |= v.target.cov_hash != nullptr;
    *any_lit |= (v.quads.color_mode == LR_COLOR_LIT && v.quads.num_quads > 0);
  }
}

static lr_status prepare(lr_ctx* ctx, int32_t n_views, const lr_view* views, void* workspace,
                         size_t workspace_bytes, Prepared* P) {
  if (n_views <= 0 || !views) return fail(ctx, LR_ERR_INVALID_ARG, "need at least one view%s");
  if (!workspace || !aligned(workspace, 256)) return fail(ctx, LR_ERR_INVALID_ARG, "workspace must be non-null and 256-byte aligned%s");
  for (int i = 0; i < n_views; ++i) {
    lr_status s = check_view(ctx, views[i]);
    if (s != LR_OK) return s;
    if ((ctx->cfg.flags & LR_FLAG_ALPHA_THRESHOLD) && (views[i].target.frag_count || views[i].target.cov_hash))
      return fail(ctx, LR_ERR_UNSUPPORTED, "fragment counts and coverage hashes need the exact composite%s");
  }
  // the batch's sorter capacity: every view's own (lr_view.sorter_k) or the context's
  P->variant = ctx->variant;
  for (int i = 0; i < n_views; ++i) {
    const int k = views[i].sorter_k ? views[i].sorter_k : ctx->cfg.sorter_k;
    int vi = -1;
    for (int j = 0; j < (int)(sizeof(kVariants) / sizeof(kVariants[0])); ++j)
      if (kVariants[j].k == k) vi = j;
    if (vi < 0) return fail(ctx, LR_ERR_INVALID_ARG, "sorter_k must be one of 1, 2, 3, 4, 6, 8, 12%s");
    if (i > 0 && vi != P->variant) return fail(ctx, LR_ERR_INVALID_ARG, "all views of a batch need the same sorter_k%s");
    P->variant = vi;
  }
  lr_status s = layout_for(ctx, n_views, views, &P->L);
  if (s != LR_OK) return s;
  set_capacity(P->L, workspace_bytes);
  if (P->L.refs_cap < 1024) return fail(ctx, LR_ERR_OOM, "workspace too small (see lr_workspace_size)%s");
  describe_views(n_views, views, P->vd, &P->any_vertex, &P->any_hash, &P->any_lit, ctx->light, ctx->bin_log2);
  if (P->any_lit && (P->any_hash || (ctx->cfg.flags & LR_FLAG_ALPHA_THRESHOLD)))
    return fail(ctx, LR_ERR_UNSUPPORTED, "lit colours with coverage hashes or the alpha threshold%s");
  P->ws = make_ws(P->L, workspace, n_views);
  P->views_dev = reinterpret_cast<ViewDev*>(static_cast<char*>(workspace) + P->L.views);
  return LR_OK;
}

// The launch sequence. View descriptors come from kernel parameters (k_write_views) or,
// when staging is given, from a copy out of pinned host memory (graph replays).
static lr_status launch_sequence(lr_ctx* ctx, const Prepared& P, cudaStream_t st, const BwdArgs* bwd, bool timed,
                                 const ViewDev* staging) {
  const Layout& L = P.L;
  Ws ws = P.ws;
  if (bwd) {
    ws.fwd = bwd->fwd;
    ws.grad_out = bwd->grad_out;
    ws.grad_col = bwd->grad_colors;
    ws.bwd_mask = bwd->exact_mask;
  }
  const int n_views = ws.n_views;
  const bool pdl = ctx->pdl_override >= 0 ? ctx->pdl_override != 0 : (ctx->cfg.flags & LR_FLAG_NO_PDL) == 0;
  rec(ctx, timed, 0, st);
  // the first kViewsPerLaunch descriptors travel with k_init, further ones with k_write_views
  ViewChunk chunk;
  memset(&chunk, 0, sizeof(chunk));
  if (staging) {
    cudaError_t e = cudaMemcpyAsync(P.views_dev, staging, sizeof(ViewDev) * (size_t)n_views, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "view descriptor copy");
  } else {
    chunk.count = std::min(kViewsPerLaunch, n_views);
    for (int i = 0; i < chunk.count; ++i) chunk.v[i] = P.vd[i];
    for (int first = kViewsPerLaunch; first < n_views; first += kViewsPerLaunch) {
      ViewChunk more;
      memset(&more, 0, sizeof(more));
      more.first = first;
      more.count = std::min(kViewsPerLaunch, n_views - first);
      for (int i = 0; i < more.count; ++i) more.v[i] = P.vd[first + i];
      launch_pdl(pdl, k_write_views, dim3(1), dim3(32), 0, st, more, P.views_dev);
    }
  }
  launch_pdl(pdl, k_init, dim3(std::max(1, (L.total_bins + 255) / 256)), dim3(256), 0, st, ws,
             (unsigned long long)L.refs_cap, chunk, P.views_dev);
  if (L.total_quads > 0) launch_pdl(pdl, k_setup, dim3((unsigned)((L.total_quads + 255) / 256)), dim3(256), 0, st, ws);
  rec(ctx, timed, 1, st);
  if (L.total_chunks > 0) launch_pdl(pdl, k_bin_count, dim3(L.total_chunks), dim3(kBinThreads), 0, st, ws);
  rec(ctx, timed, 2, st);
  launch_pdl(pdl, k_bin_scan, dim3(1), dim3(1024), 0, st, ws);
  rec(ctx, timed, 3, st);
  if (L.total_chunks > 0) launch_pdl(pdl, k_bin_scatter, dim3(L.total_chunks), dim3(kBinThreads), 0, st, ws);
  rec(ctx, timed, 4, st);
  launch_pdl(pdl, k_bin_sort, dim3(L.total_bins), dim3(256), kSortSmemBytes, st, ws);
  launch_pdl(pdl, k_bin_sort_big, dim3(ctx->sms), dim3(kSortBigThreads), kSortBigSmemBytes, st, ws);
  rec(ctx, timed, 5, st);
  const bool carry = P.any_vertex || P.any_lit || (ctx->cfg.flags & LR_FLAG_CARRY_COLORS);
  const bool ath = !bwd && (ctx->cfg.flags & LR_FLAG_ALPHA_THRESHOLD);   // no hash then (prepare)
  // (lit views: neither hash nor threshold, see prepare)
  const int mode = bwd ? 2 : (P.any_lit ? 17 : ((carry ? 1 : 0) | (P.any_hash ? 4 : 0) | (ath ? 8 : 0)));
  ws.t_min = ath ? kAlphaTMin : 0.0f;
  const VariantState& VS = ctx->vs[P.variant];
  // the strip kernel (32-pixel bins) or 8x8 blocks for forward exact renders of flat or
  // carried colours, when asked for and built
  const bool strip = ctx->cfg.shared_setup && VS.v->launch_strip && !bwd && !ath && !P.any_lit &&
                     ctx->bin_log2 == kBinLog2Default;
  const bool blk8 = !strip && ctx->cfg.block_h == 8 && VS.v->launch8 && !bwd && !ath && !P.any_lit;
  cudaError_t e;
  if (strip) {
    e = VS.v->launch_strip(mode, ws, ctx->sms * (carry ? VS.vtx_s : VS.flat_s), st);
  } else if (blk8) {
    e = VS.v->launch8(mode, ws, ctx->sms * (carry ? VS.vtx8 : VS.flat8), st);
  } else {
    const int rblocks = bwd ? VS.bwd : (P.any_lit ? VS.lit : (carry ? VS.vtx : VS.flat));
    e = VS.v->launch(mode, ws, ctx->sms * rblocks, st);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "raster launch");
  rec(ctx, timed, 6, st);
  e = launch_overflow(bwd != nullptr, ws, ctx->sms * ctx->ovf_blocks, st, pdl);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "overflow launch");
  rec(ctx, timed, 7, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
  return LR_OK;
}

static void remember_last(lr_ctx* ctx, const Prepared& P, cudaStream_t st, void* workspace, bool timed) {
  ctx->last_stream = st;
  ctx->last_ws = workspace;
  ctx->last_views = P.ws.n_views;
  ctx->last_quads = P.L.total_quads;
  ctx->last_cap = P.L.refs_cap;
  ctx->have_last = true;
  ctx->last_timed = timed;
}

static lr_status enqueue(lr_ctx* ctx, int32_t n_views, const lr_view* views, void* workspace,
                         size_t workspace_bytes, lr_stream stream, const BwdArgs* bwd) {
  if (!ctx) return LR_ERR_INVALID_ARG;
  Prepared P;
  lr_status s = prepare(ctx, n_views, views, workspace, workspace_bytes, &P);
  if (s != LR_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const bool timed = (ctx->cfg.flags & LR_FLAG_TIMING) != 0;
  s = launch_sequence(ctx, P, st, bwd, timed, nullptr);
  if (s != LR_OK) return s;
  remember_last(ctx, P, st, workspace, timed);
  return LR_OK;
}

// ---- captured batches (CUDA graphs) ------------------------------------------------------

struct lr_graph {
  lr_ctx* ctx = nullptr;
  void* ws = nullptr;
  size_t bytes = 0;
  Prepared P;
  std::vector<lr_view> shape;        // the views the graph was made for
  ViewDev* staging[2] = {nullptr, nullptr};   // pinned; read by each replay's first node
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool launched[2] = {false, false};
  int next = 0;
};

static void free_graph(lr_graph* g) {
  for (int b = 0; b < 2; ++b) {
    if (g->done[b]) { cudaEventSynchronize(g->done[b]); cudaEventDestroy(g->done[b]); }
    if (g->exec[b]) cudaGraphExecDestroy(g->exec[b]);
    if (g->staging[b]) cudaFreeHost(g->staging[b]);
  }
  delete g;
}

extern "C" lr_status lr_graph_create(lr_ctx* ctx, int32_t n_views, const lr_view* views, void* workspace,
                                     size_t workspace_bytes, lr_graph** out) {
  if (!ctx || !out) return LR_ERR_INVALID_ARG;
  *out = nullptr;
  lr_graph* g = new (std::nothrow) lr_graph();
  if (!g) return LR_ERR_OOM;
  g->ctx = ctx;
  g->ws = workspace;
  g->bytes = workspace_bytes;
  lr_status s = prepare(ctx, n_views, views, workspace, workspace_bytes, &g->P);
  if (s != LR_OK) { delete g; return s; }
  g->shape.assign(views, views + n_views);
  cudaError_t e = cudaSetDevice(ctx->device);
  cudaStream_t cap = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMallocHost(reinterpret_cast<void**>(&g->staging[b]), sizeof(ViewDev) * (size_t)n_views);
    if (e != cudaSuccess) break;
    memcpy(g->staging[b], g->P.vd.data(), sizeof(ViewDev) * (size_t)n_views);
    e = cudaEventCreateWithFlags(&g->done[b], cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    s = launch_sequence(ctx, g->P, cap, nullptr, false, g->staging[b]);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
    if (s != LR_OK || ee != cudaSuccess) { e = ee != cudaSuccess ? ee : cudaErrorUnknown; if (graph) cudaGraphDestroy(graph); break; }
    e = cudaGraphInstantiate(&g->exec[b], graph, 0);
    cudaGraphDestroy(graph);
  }
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess || s != LR_OK) {
    lr_status r = s != LR_OK ? s : cuda_fail(ctx, e, "graph capture");
    free_graph(g);
    return r;
  }
  *out = g;
  return LR_OK;
}

extern "C" lr_status lr_graph_launch(lr_graph* g, const lr_view* views, lr_stream stream) {
  if (!g) return LR_ERR_INVALID_ARG;
  lr_ctx* ctx = g->ctx;
  const int n = g->P.ws.n_views;
  const int b = g->next;
  if (g->launched[b]) {
    // the replay that last read this staging buffer must have copied it
    cudaError_t e = cudaEventSynchronize(g->done[b]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize");
  }
  if (views) {
    for (int i = 0; i < n; ++i) {
      const lr_view& a = views[i];
      const lr_view& s0 = g->shape[i];
      if (a.width != s0.width || a.height != s0.height || a.quads.num_quads != s0.quads.num_quads ||
          a.quads.color_mode != s0.quads.color_mode || (a.target.cov_hash == nullptr) != (s0.target.cov_hash == nullptr) ||
          (a.sorter_k ? a.sorter_k : ctx->cfg.sorter_k) != (s0.sorter_k ? s0.sorter_k : ctx->cfg.sorter_k))
        return fail(ctx, LR_ERR_INVALID_ARG, "graph launch views must keep the captured shapes%s");
      lr_status s = check_view(ctx, a);
      if (s != LR_OK) return s;
    }
    std::vector<ViewDev> vd;
    bool any_vertex = false, any_hash = false, any_lit = false;
    // replays keep the light the graph was captured with
    describe_views(n, views, vd, &any_vertex, &any_hash, &any_lit, g->P.vd[0].light, ctx->bin_log2);
    memcpy(g->staging[b], vd.data(), sizeof(ViewDev) * (size_t)n);
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGraphLaunch(g->exec[b], st);
  if (e == cudaSuccess) e = cudaEventRecord(g->done[b], st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
  g->launched[b] = true;
  g->next = b ^ 1;
  remember_last(ctx, g->P, st, g->ws, false);
  return LR_OK;
}

extern "C" lr_status lr_graph_destroy(lr_graph* g) {
  if (!g) return LR_ERR_INVALID_ARG;
  free_graph(g);
  return LR_OK;
}

extern "C" lr_status lr_render_batch(lr_ctx* ctx, int32_t n_views, const lr_view* views, void* workspace,
                                     size_t workspace_bytes, lr_stream stream) {
  return enqueue(ctx, n_views, views, workspace, workspace_bytes, stream, nullptr);
}

extern "C" lr_status lr_render_backward(lr_ctx* ctx, const lr_quads* quads, const lr_camera* camera,
                                        int32_t width, int32_t height, const float* fwd_rgba,
                                        const float* grad_out, const uint32_t* exact_mask,
                                        float* grad_colors, void* workspace, size_t workspace_bytes,
                                        lr_stream stream) {
  if (!ctx) return LR_ERR_INVALID_ARG;
  if (!quads || !camera || !fwd_rgba || !grad_out || !grad_colors)
    return fail(ctx, LR_ERR_INVALID_ARG, "null argument%s");
  if (quads->num_quads > 0 && quads->color_mode != LR_COLOR_FLAT)
    return fail(ctx, LR_ERR_UNSUPPORTED, "the backward pass supports flat per-quad colours only%s");
  if (ctx->cfg.flags & LR_FLAG_ALPHA_THRESHOLD)
    return fail(ctx, LR_ERR_UNSUPPORTED, "no backward pass for the alpha-threshold composite%s");
  if (!aligned(fwd_rgba, 16) || !aligned(grad_out, 16) || !aligned(grad_colors, 16))
    return fail(ctx, LR_ERR_INVALID_ARG, "fwd_rgba, grad_out and grad_colors must be 16-byte aligned%s");
  lr_view v;
  memset(&v, 0, sizeof(v));
  v.quads = *quads;
  v.camera = *camera;
  v.width = width;
  v.height = height;
  v.target.rgba = const_cast<float*>(fwd_rgba);   // not written by the backward pass
  if (exact_mask && !aligned(exact_mask, 4)) return fail(ctx, LR_ERR_INVALID_ARG, "exact_mask must be 4-byte aligned%s");
  BwdArgs b{fwd_rgba, grad_out, grad_colors, exact_mask};
  return enqueue(ctx, 1, &v, workspace, workspace_bytes, stream, &b);
}

extern "C" lr_status lr_render(lr_ctx* ctx, const lr_quads* quads, const lr_camera* camera, int32_t width,
                               int32_t height, float* out_rgba, void* workspace, size_t workspace_bytes,
                               lr_stream stream) {
  if (!ctx) return LR_ERR_INVALID_ARG;
  if (!quads || !camera) return fail(ctx, LR_ERR_INVALID_ARG, "null quads or camera%s");
  lr_view v;
  memset(&v, 0, sizeof(v));
  v.quads = *quads;
  v.camera = *camera;
  v.width = width;
  v.height = height;
  v.target.rgba = out_rgba;
  return lr_render_batch(ctx, 1, &v, workspace, workspace_bytes, stream);
}

// ---- multisampling --------------------------------------------------------------------

namespace lr {

constexpr int kMaxSamples = 16;

// default sample patterns, offsets from the pixel centre in 1/256 px: 4 samples on a grid
// rotated so that each has its own row and column (offsets +-1/8 and +-3/8 px); 16 samples
// one per row and column of a 16x16 sub-grid, row i (from the top) in column (5 i + 3) mod 16
static void default_samples(int n, int off[][2]) {
  if (n == 4) {
    static const int r4[4][2] = {{-32, -96}, {96, -32}, {-96, 32}, {32, 96}};
    for (int i = 0; i < 4; ++i) { off[i][0] = r4[i][0]; off[i][1] = r4[i][1]; }
  } else {
    for (int i = 0; i < 16; ++i) {
      off[i][0] = 16 * ((5 * i + 3) % 16) - 120;
      off[i][1] = 16 * i - 120;
    }
  }
}

// out = (sum of the n sample images, in sample order) / n, per channel in fp32
__global__ void k_resolve(const float4* samples, int n, long long npix, float4* out) {
  pdl_begin();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= npix) return;
  float4 acc = samples[i];
  for (int s = 1; s < n; ++s) {
    const float4 v = samples[(long long)s * npix + i];
    acc.x = __fadd_rn(acc.x, v.x);
    acc.y = __fadd_rn(acc.y, v.y);
    acc.z = __fadd_rn(acc.z, v.z);
    acc.w = __fadd_rn(acc.w, v.w);
  }
  const float fn = (float)n;
  out[i] = make_float4(__fdiv_rn(acc.x, fn), __fdiv_rn(acc.y, fn), __fdiv_rn(acc.z, fn), __fdiv_rn(acc.w, fn));
}

static size_t msaa_image_bytes(int n, int width, int height) {
  return align256(sizeof(float4) * (size_t)width * (size_t)height * (size_t)n);
}

}  // namespace lr

extern "C" lr_status lr_workspace_size_msaa(const lr_ctx* ctx, int64_t num_quads, int32_t width, int32_t height,
                                            int32_t n_samples, size_t* out_bytes) {
  if (!ctx || !out_bytes || num_quads < 0 || width <= 0 || height <= 0) return LR_ERR_INVALID_ARG;
  if (n_samples < 1 || n_samples > kMaxSamples) return LR_ERR_INVALID_ARG;
  if (width > ctx->cfg.max_width || height > ctx->cfg.max_height) return LR_ERR_TOO_LARGE;
  std::vector<long long> Q(n_samples, num_quads);
  std::vector<int> W(n_samples, width), H(n_samples, height);
  Layout L = make_layout(n_samples, Q.data(), W.data(), H.data(), ctx->bin_log2);
  if (L.total_quads > 0x7FFFFFFFLL || L.total_pix > 0xFFFFFFFFLL) return LR_ERR_TOO_LARGE;
  *out_bytes = msaa_image_bytes(n_samples, width, height) + bytes_for_refs(L, default_refs(L, ctx->cfg.ref_factor));
  return LR_OK;
}

extern "C" lr_status lr_render_msaa(lr_ctx* ctx, const lr_quads* quads, const lr_camera* camera, int32_t width,
                                    int32_t height, int32_t n_samples, const int32_t* sample_offsets, float* out_rgba,
                                    void* workspace, size_t workspace_bytes, lr_stream stream) {
  if (!ctx) return LR_ERR_INVALID_ARG;
  if (!quads || !camera || !out_rgba) return fail(ctx, LR_ERR_INVALID_ARG, "null quads, camera or output%s");
  if (n_samples < 1 || n_samples > kMaxSamples) return fail(ctx, LR_ERR_INVALID_ARG, "n_samples must be 1..16%s");
  if (!sample_offsets && n_samples != 4 && n_samples != 16)
    return fail(ctx, LR_ERR_INVALID_ARG, "default sample patterns exist for 4 and 16 samples only%s");
  if (width <= 0 || height <= 0) return fail(ctx, LR_ERR_INVALID_ARG, "width and height must be positive%s");
  if (!aligned(out_rgba, 16)) return fail(ctx, LR_ERR_INVALID_ARG, "out_rgba must be 16-byte aligned%s");
  if (!workspace || !aligned(workspace, 256))
    return fail(ctx, LR_ERR_INVALID_ARG, "workspace must be non-null and 256-byte aligned%s");
  int off[kMaxSamples][2];
  if (sample_offsets) {
    for (int i = 0; i < n_samples; ++i) {
      off[i][0] = sample_offsets[2 * i];
      off[i][1] = sample_offsets[2 * i + 1];
      if (off[i][0] < -127 || off[i][0] > 127 || off[i][1] < -127 || off[i][1] > 127)
        return fail(ctx, LR_ERR_INVALID_ARG, "sample offsets must lie in [-127, 127]%s");
    }
  } else {
    default_samples(n_samples, off);
  }
  const size_t img = msaa_image_bytes(n_samples, width, height);
  if (workspace_bytes <= img) return fail(ctx, LR_ERR_OOM, "workspace too small (see lr_workspace_size_msaa)%s");
  float4* samples = static_cast<float4*>(workspace);
  const long long npix = (long long)width * height;
  std::vector<lr_view> views(n_samples);
  for (int i = 0; i < n_samples; ++i) {
    lr_view& v = views[i];
    memset(&v, 0, sizeof(v));
    v.quads = *quads;
    v.camera = *camera;
    v.width = width;
    v.height = height;
    v.target.rgba = reinterpret_cast<float*>(samples + (long long)i * npix);
  }
  void* ws = static_cast<char*>(workspace) + img;
  Prepared P;
  lr_status s = prepare(ctx, n_samples, views.data(), ws, workspace_bytes - img, &P);
  if (s != LR_OK) return s;
  for (int i = 0; i < n_samples; ++i) {
    P.vd[i].sub_x = off[i][0];
    P.vd[i].sub_y = off[i][1];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  const bool timed = (ctx->cfg.flags & LR_FLAG_TIMING) != 0;
  s = launch_sequence(ctx, P, st, nullptr, timed, nullptr);
  if (s != LR_OK) return s;
  const bool pdl = (ctx->cfg.flags & LR_FLAG_NO_PDL) == 0;
  e = launch_pdl(pdl, k_resolve, dim3((unsigned)((npix + 255) / 256)), dim3(256), 0, st,
                 static_cast<const float4*>(samples), (int)n_samples, npix, reinterpret_cast<float4*>(out_rgba));
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "resolve launch");
  remember_last(ctx, P, st, ws, timed);
  return LR_OK;
}

extern "C" lr_status lr_get_stats(lr_ctx* ctx, lr_stats* stats) {
  if (!ctx) return LR_ERR_INVALID_ARG;
  if (!ctx->have_last) return fail(ctx, LR_ERR_INVALID_ARG, "no render issued on this context%s");
  cudaError_t e = cudaStreamSynchronize(ctx->last_stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
  e = cudaMemcpy(ctx->host_ctrl, ctx->last_ws, sizeof(Ctrl), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(ctrl)");
  const Ctrl& h = *ctx->host_ctrl;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->status = h.error;
    stats->n_views = ctx->last_views;
    stats->quads_in = ctx->last_quads;
    // k_setup counts culled quads only; every other input quad is visible
    int64_t culled = 0;
    for (int i = 0; i < 8; ++i) {
      stats->culled[i] = (int64_t)h.culled[i];
      culled += stats->culled[i];
    }
    stats->quads_visible = ctx->last_quads - culled;
    stats->bin_refs = (int64_t)h.refs_total;
    stats->bin_refs_capacity = ctx->last_cap;
    stats->bins_nonempty = (int64_t)h.bins_nonempty;
    stats->bins_high = (int64_t)h.bins_high;
    stats->max_bin_refs = (int64_t)h.max_bin;
    stats->fragments = (int64_t)h.fragments;
    stats->overflow_pixels = (int64_t)h.ovf_count;
    for (int i = 0; i < 3; ++i) stats->sort_bins[i] = (int64_t)h.sort_branch[i];
    if (ctx->last_timed) {
      for (int i = 0; i < 7; ++i) cudaEventElapsedTime(&stats->stage_ms[i], ctx->ev[i], ctx->ev[i + 1]);
      cudaEventElapsedTime(&stats->stage_ms[7], ctx->ev[0], ctx->ev[7]);
    }
  }
  if (h.error != 0) {
    snprintf(ctx->err, sizeof(ctx->err), "device reported status %d (%s)", h.error,
             h.error == LR_ERR_OVERFLOW ? "bin-reference capacity exceeded"
                                        : h.error == LR_ERR_INVALID_ARG ? "vertex index out of range" : "error");
    return (lr_status)h.error;
  }
  return LR_OK;
}

extern "C" const char* lr_last_error(const lr_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err;
}
