// lr_noalloc.cu -- lr_render_noalloc: a render entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need a frame: a
// plugin called per frame by a host engine that owns all device memory through its own
// pool and forbids cudaMalloc after start-up (a cudaMalloc there can stall every stream
// of the process and can fail under the host's memory budget), or code that must not
// block at all while other work is in flight. They cannot provide the workspace that
// lr_render takes either. This entry point runs the same pipeline kernels, with the same
// sorter capacity (K = 3) as the default context, on a scratch area that is a file-scope
// device array of LR_NOALLOC_SCRATCH_BYTES bytes, instead of a caller-provided
// workspace. The array is part of the library's device code: every GPU on which the
// library's device code is loaded holds it until the process exits.
//
// Set-up: the first call on each device (with that device current) looks up the array's
// device address with cudaGetSymbolAddress, checks the return code, and sets the kernel
// attributes; later calls on that device reuse the cached address. Make that first call
// before any stream capture. No call allocates memory (no cudaMalloc, cudaFree,
// cudaMallocHost, no PyTorch allocator, no host heap).
//
// Every call shares the one array and leaves its contents behind: the pipeline's first
// kernel zeroes the counters and the control block each call, everything else is fully
// overwritten. Calls whose GPU work overlaps (different streams, or a call issued while a
// previous one is still running on another stream) race on the array and produce garbage.
#include <cstring>
#include <mutex>

#include "lr_common.cuh"
#include "lr_raster.cuh"

namespace lr {
__global__ void k_init(Ws ws, unsigned long long refs_cap, ViewChunk views, ViewDev* views_dst);
__global__ void k_setup(Ws ws);
__global__ void k_bin_count(Ws ws);
__global__ void k_bin_scan(Ws ws);
__global__ void k_bin_scatter(Ws ws);
__global__ void k_bin_sort(Ws ws);
__global__ void k_bin_sort_big(Ws ws);
cudaError_t prepare_raster_3(int* blocks_flat, int* blocks_vtx, int* blocks_bwd, int* blocks_lit);
cudaError_t launch_raster_3(int mode, const Ws& ws, int grid, cudaStream_t st);
cudaError_t overflow_occupancy(int* blocks_per_sm);
cudaError_t launch_overflow(bool bwd, const Ws& ws, int grid, cudaStream_t st, bool pdl);
}  // namespace lr

using namespace lr;

static __device__ __align__(256) unsigned char g_noalloc_scratch[LR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool ready = false;
  unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch
  int sms = 0, blocks_flat = 1, blocks_vtx = 1, ovf_blocks = 1;
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

__global__ void k_noalloc_view(ViewDev v, ViewDev* dst) { *dst = v; }

__global__ void k_noalloc_status(const Ctrl* ctrl, int32_t* out) { *out = ctrl->error; }

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" lr_status lr_render_noalloc(const lr_quads* quads, const lr_camera* camera, int32_t width,
                                       int32_t height, float* out_rgba, int32_t* device_status,
                                       lr_stream stream) {
  if (!quads || !camera || !out_rgba) return LR_ERR_INVALID_ARG;
  if (width <= 0 || height <= 0) return LR_ERR_INVALID_ARG;
  if (width > 65535 || height > 65535) return LR_ERR_TOO_LARGE;
  const lr_quads& q = *quads;
  if (q.num_quads < 0 || q.num_vertices < 0) return LR_ERR_INVALID_ARG;
  if (q.num_quads > 0) {
    if (!q.positions || !q.colors) return LR_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(q.positions) & 15) || (reinterpret_cast<uintptr_t>(q.colors) & 15) ||
        (q.indices && (reinterpret_cast<uintptr_t>(q.indices) & 15)))
      return LR_ERR_INVALID_ARG;
    if (q.color_mode != LR_COLOR_FLAT && q.color_mode != LR_COLOR_VERTEX) return LR_ERR_INVALID_ARG;
  }
  if (reinterpret_cast<uintptr_t>(out_rgba) & 15) return LR_ERR_INVALID_ARG;
  if (device_status && (reinterpret_cast<uintptr_t>(device_status) & 3)) return LR_ERR_INVALID_ARG;
  if (!(camera->near_z > 0.0f) || !(camera->far_z >= camera->near_z) || !(camera->far_z < 3.4e38f))
    return LR_ERR_INVALID_ARG;

  // ---- scratch layout (sizes must fit the static array) --------------------------------
  const long long Q = q.num_quads;
  constexpr int kB = 1 << kBinLog2Default;   // 32-pixel bins, the default context's
  const int nbx = (width + kB - 1) / kB, nby = (height + kB - 1) / kB;
  const long long nbins = (long long)nbx * nby, npix = (long long)width * height;
  size_t o = 0;
  const size_t o_ctrl = o; o = up256(o + sizeof(Ctrl));
  const size_t o_view = o; o = up256(o + sizeof(ViewDev));
  const bool vtx = q.color_mode == LR_COLOR_VERTEX;
  const size_t o_rec = o; o = up256(o + 64 * (size_t)Q);
  const size_t o_rect = o; o = up256(o + 8 * (size_t)Q);
  const size_t o_info = o; o = up256(o + 4 * (size_t)Q);
  const size_t o_rep = o; o = up256(o + 4 * (size_t)Q);
  const size_t o_cnt = o; o = up256(o + 4 * (size_t)nbins);
  const size_t o_off = o; o = up256(o + 4 * ((size_t)nbins + 1));
  const size_t o_cur = o; o = up256(o + 4 * (size_t)nbins);
  const size_t o_span = o; o = up256(o + 8 * (size_t)((Q + kChunkQuads - 1) / kChunkQuads));
  const size_t o_ord = o; o = up256(o + 4 * (size_t)nbins);
  const size_t o_ovf = o; o = up256(o + 4 * (size_t)npix);
  if (o >= (size_t)LR_NOALLOC_SCRATCH_BYTES) return LR_ERR_TOO_LARGE;
  // per reference 8 B key + 8 B merge slot + 4 B bitmap word, plus 32 bitmap words per bin
  const size_t fixed_hb = 128 * (size_t)nbins + 2048;
  if (o + fixed_hb >= (size_t)LR_NOALLOC_SCRATCH_BYTES) return LR_ERR_TOO_LARGE;
  long long cap = (long long)(((size_t)LR_NOALLOC_SCRATCH_BYTES - o - fixed_hb) / 20) & ~63LL;
  if (cap > 0xFFFFFF00LL) cap = 0xFFFFFF00LL;
  // require room for at least two references per quad and one per bin
  if (cap < 2 * Q + nbins + 1024) return LR_ERR_TOO_LARGE;
  const size_t o_refs = o;
  const size_t o_tmp = up256(o_refs + 8 * (size_t)cap);
  const size_t o_hb = up256(o_tmp + 8 * (size_t)cap);

  // ---- per-device set-up (first call on this device only) ------------------------------
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LR_ERR_CUDA;
  DeviceSetup ds;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup& d = g_setup[dev];
    if (!d.ready) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LR_ERR_CUDA;
      int blocks_bwd = 1, blocks_lit = 1;
      if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          prepare_raster_3(&d.blocks_flat, &d.blocks_vtx, &blocks_bwd, &blocks_lit) != cudaSuccess ||
          overflow_occupancy(&d.ovf_blocks) != cudaSuccess ||
          cudaFuncSetAttribute(k_bin_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSortSmemBytes) != cudaSuccess ||
          cudaFuncSetAttribute(k_bin_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSortBigSmemBytes) != cudaSuccess)
        return LR_ERR_CUDA;
      // Load every kernel this entry point can launch now, not at its first launch: with
      // CUDA's lazy module loading a kernel's first launch loads it, which a later call
      // made under stream capture must not do (e.g. a first call without device_status,
      // then a captured call with one). cudaFuncGetAttributes forces the load.
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, k_noalloc_view) != cudaSuccess ||
          cudaFuncGetAttributes(&fa, k_noalloc_status) != cudaSuccess ||
          cudaFuncGetAttributes(&fa, k_init) != cudaSuccess || cudaFuncGetAttributes(&fa, k_setup) != cudaSuccess ||
          cudaFuncGetAttributes(&fa, k_bin_count) != cudaSuccess ||
          cudaFuncGetAttributes(&fa, k_bin_scan) != cudaSuccess ||
          cudaFuncGetAttributes(&fa, k_bin_scatter) != cudaSuccess)
        return LR_ERR_CUDA;
      d.scratch = static_cast<unsigned char*>(p);
      d.blocks_flat = d.blocks_flat > 0 ? d.blocks_flat : 1;
      d.blocks_vtx = d.blocks_vtx > 0 ? d.blocks_vtx : 1;
      d.ovf_blocks = d.ovf_blocks > 0 ? d.ovf_blocks : 1;
      d.ready = true;
    }
    ds = d;
  }

  // ---- view descriptor and workspace pointers ------------------------------------------
  ViewDev v;
  memset(&v, 0, sizeof(v));
  v.pos = q.positions;
  v.idx = q.indices;
  v.col = q.colors;
  v.out = out_rgba;
  for (int k = 0; k < 4; ++k) {
    v.m[k] = camera->view_proj[k];
    v.m[4 + k] = camera->view_proj[4 + k];
    v.m[8 + k] = camera->view_proj[12 + k];
  }
  v.near_z = camera->near_z;
  v.far_z = camera->far_z;
  v.half_w = 0.5f * (float)width;
  v.half_h = 0.5f * (float)height;
  v.num_vertices = q.num_vertices;
  v.num_quads = (int)Q;
  v.color_mode = q.color_mode;
  v.width = width;
  v.height = height;
  v.nbx = nbx;
  v.nby = nby;
  unsigned char* base = ds.scratch;
  Ws ws;
  memset(&ws, 0, sizeof(ws));
  ws.ctrl = reinterpret_cast<Ctrl*>(base + o_ctrl);
  ws.views = reinterpret_cast<const ViewDev*>(base + o_view);
  ws.n_views = 1;
  ws.total_bins = (int)nbins;
  ws.total_quads = Q;
  ws.total_pix = npix;
  ws.refs_cap = cap;
  ws.bin_log2 = kBinLog2Default;
  ws.rec = reinterpret_cast<int4*>(base + o_rec);
  ws.rec_rect = reinterpret_cast<uint2*>(base + o_rect);
  ws.rec_info = reinterpret_cast<uint32_t*>(base + o_info);
  ws.rec_rep = reinterpret_cast<float*>(base + o_rep);
  ws.bin_count = reinterpret_cast<uint32_t*>(base + o_cnt);
  ws.bin_off = reinterpret_cast<uint32_t*>(base + o_off);
  ws.bin_cursor = reinterpret_cast<uint32_t*>(base + o_cur);
  ws.chunk_span = reinterpret_cast<uint2*>(base + o_span);
  ws.bin_order = reinterpret_cast<uint32_t*>(base + o_ord);
  ws.refs = reinterpret_cast<unsigned long long*>(base + o_refs);
  ws.refs_tmp = reinterpret_cast<unsigned long long*>(base + o_tmp);
  ws.ref_hb = reinterpret_cast<uint32_t*>(base + o_hb);
  ws.ovf_list = reinterpret_cast<uint32_t*>(base + o_ovf);

  // ---- the pipeline, as lr_render launches it ------------------------------------------
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int chunks = (int)((Q + kChunkQuads - 1) / kChunkQuads);
  k_noalloc_view<<<1, 1, 0, st>>>(v, reinterpret_cast<ViewDev*>(base + o_view));
  ViewChunk no_views;
  memset(&no_views, 0, sizeof(no_views));
  k_init<<<(int)((nbins + 255) / 256), 256, 0, st>>>(ws, (unsigned long long)cap, no_views, nullptr);
  if (Q > 0) k_setup<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(ws);
  if (chunks > 0) k_bin_count<<<chunks, kBinThreads, 0, st>>>(ws);
  k_bin_scan<<<1, 1024, 0, st>>>(ws);
  if (chunks > 0) k_bin_scatter<<<chunks, kBinThreads, 0, st>>>(ws);
  k_bin_sort<<<(int)nbins, 256, kSortSmemBytes, st>>>(ws);
  k_bin_sort_big<<<ds.sms, kSortBigThreads, kSortBigSmemBytes, st>>>(ws);
  const bool vtx_kernel = Q > 0 && vtx;
  if (launch_raster_3(vtx_kernel ? 1 : 0, ws, ds.sms * (vtx_kernel ? ds.blocks_vtx : ds.blocks_flat), st) != cudaSuccess)
    return LR_ERR_CUDA;
  if (launch_overflow(false, ws, ds.sms * ds.ovf_blocks, st, false) != cudaSuccess) return LR_ERR_CUDA;
  if (device_status) k_noalloc_status<<<1, 1, 0, st>>>(ws.ctrl, device_status);
  return cudaGetLastError() == cudaSuccess ? LR_OK : LR_ERR_CUDA;
}
