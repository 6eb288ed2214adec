// lr_overflow.cu -- k_overflow, the exact fallback for the pixels whose order the
// fixed-size per-pixel sorter could not guarantee and that the rasteriser registered. The
// paper detects such pixels by growing the depth filter by one and suggests recording them
// and redoing them afterwards with a slower exact method, which it leaves unbuilt (Sec. 2,
// "Sample blending"; Sec. 3, "Fragment sorting errors"). One warp per registered pixel
// (overflow_pixel, lr_exact.cuh); the pixels of a frame are few and run in one wave, so the
// kernel's time is about one warp's chain of dependent loads.
#include "lr_raster.cuh"
#include "lr_exact.cuh"

namespace lr {

#ifndef LR_OVF_BUF
#define LR_OVF_BUF 512
#endif
// per-warp buffer of the exact path (a power of two; a pass composites 15/32 of it): 512
// entries (4 KB) let seven CTAs of four warps share an SM (registers and shared memory), so
// up to 4,256 registered pixels of a frame run in one wave, one warp each
constexpr int kExactBuf = LR_OVF_BUF;

// the exact path over the registered pixel list
template <bool BWD>
__global__ __launch_bounds__(kOvfThreads, BWD ? 5 : 7) void k_overflow(Ws ws) {
  pdl_begin();
  __shared__ unsigned long long sbuf[kOvfThreads / 32][kExactBuf];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (ws.ctrl->error == LR_ERR_OVERFLOW) return;
  const unsigned long long total = ws.ctrl->ovf_count;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&ws.ctrl->ovf_head, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    overflow_pixel<BWD, kExactBuf>(ws, (long long)ws.ovf_list[item], sbuf[warp]);
  }
}

cudaError_t overflow_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_overflow<false>, kOvfThreads, 0);
}

cudaError_t launch_overflow(bool bwd, const Ws& ws, int grid, cudaStream_t st, bool pdl) {
  if (bwd) return launch_pdl(pdl, k_overflow<true>, dim3(grid), dim3(kOvfThreads), 0, st, ws);
  return launch_pdl(pdl, k_overflow<false>, dim3(grid), dim3(kOvfThreads), 0, st, ws);
}

}  // namespace lr
