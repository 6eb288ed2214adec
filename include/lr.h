/*
 * lr.h -- C ABI of a GB300 (sm_103a) implementation of the exact order-independent-
 * transparency quad rasteriser of "LucidRaster: GPU Software Rasterizer for Exact
 * Order-Independent Transparency" (arXiv 2405.13364).
 *
 * The pipeline is the paper's sort-middle design (Sec. 2, "Pipeline description"):
 * quad setup (Stage 1), 32x32-pixel binning (Stage 2), per-bin rasterisation with a
 * two-stage sort and blending (Stage 3), plus an exact fallback for pixels whose order
 * the fixed-size sorter cannot guarantee (Sec. 2, "Sample blending", suggests recording
 * the misordered pixels and redoing them afterwards with a slower exact method).
 *
 * Conventions for every entry point:
 *  - Plain pointers only. Pointers documented as "device" must point to memory of the
 *    context's CUDA device; "host" pointers to ordinary host memory.
 *  - The caller owns every input, output and workspace buffer; the library owns only the
 *    lr_ctx object and what it allocates internally (a small control buffer, serving
 *    state). Rendering calls are asynchronous on the given stream: they return once the
 *    work is enqueued, and the caller must keep all buffers alive and untouched until the
 *    stream has finished it.
 *  - Every function returns an lr_status and never aborts the process. Errors found
 *    while the GPU runs (capacity exceeded, out-of-range vertex indices) are recorded in
 *    the workspace and reported by lr_get_stats(), which synchronises.
 *  - Not thread-safe per context, except lr_submit / lr_poll which may be called from
 *    any thread.
 */
#ifndef LR_H_
#define LR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lr_ctx lr_ctx;            /* opaque, owned by the library */
typedef struct CUstream_st* lr_stream;   /* a cudaStream_t; NULL = the legacy default stream */

typedef enum {
  LR_OK = 0,
  LR_PENDING = 1,            /* lr_poll: the request has not finished yet */
  LR_ERR_INVALID_ARG = -1,   /* bad argument, or out-of-range vertex index found on the GPU */
  LR_ERR_TOO_LARGE = -2,     /* width/height above the context's maximum, or too many quads */
  LR_ERR_OOM = -3,           /* a device allocation failed / workspace too small */
  LR_ERR_CUDA = -4,          /* a CUDA runtime call failed (see lr_last_error) */
  LR_ERR_TIMEOUT = -5,       /* lr_poll's time limit ran out */
  LR_ERR_OVERFLOW = -6,      /* the workspace's bin-reference capacity was exceeded */
  LR_ERR_UNSUPPORTED = -7,   /* option combination not implemented */
  LR_ERR_MASK_MISMATCH = -8  /* lr_render_backward: the exact-path mask given does not
                                match this scene and context (gradients not valid) */
} lr_status;

/* Colour modes of lr_quads.colors. LR_COLOR_LIT: per-vertex colours with normals and one
 * directional light (lr_set_lighting); the paper shades its samples with a simple material
 * (Sec. 2, "Stage 3"; Sec. 4), and this is the plainest shading with normals. */
enum { LR_COLOR_FLAT = 0, LR_COLOR_VERTEX = 1, LR_COLOR_LIT = 2 };

/* lr_config.flags */
enum {
  LR_FLAG_TIMING = 1,       /* record per-stage CUDA events; lr_get_stats reports stage_ms */
  LR_FLAG_CARRY_COLORS = 2, /* flat-colour scenes too: the per-pixel sorter carries each
                               fragment's colour (fetched once per half-block) instead of
                               reading it when the fragment is blended (a tuning choice) */
  LR_FLAG_NO_PDL = 4,       /* launch without programmatic dependent launch. By default each
                               kernel of a render may be scheduled while its predecessor
                               drains (it waits for it before touching memory); a context
                               rendering on several streams at once sets this flag, since
                               such waiting kernels hold SM resources other streams need.
                               The server's own context always sets it. */
  LR_FLAG_ALPHA_THRESHOLD = 8 /* opt-in, lossy (Sec. 2 "Sample blending", Sec. 3 "Alpha
                               threshold"): a pixel stops blending once its accumulated alpha
                               reaches 1 - 1/128, i.e. each fragment is blended only while the
                               fp32 transmittance T = prod (1 - a) of the fragments in front of
                               it (in exact depth order) is above 1/128. The image then differs
                               from the exact composite by at most 1/128 per channel. Candidate
                               quads that cannot reach in front of any unfinished pixel of a
                               half-block are skipped, so lr_stats.fragments counts the
                               fragments evaluated. Renders that ask for frag_count or cov_hash
                               and lr_render_backward return LR_ERR_UNSUPPORTED on such a
                               context. */
};

/* Creation-time parameters. Zero selects the default. */
typedef struct {
  int32_t max_width;         /* default 2560 (the paper's limit is 2560x2048, Sec. 4) */
  int32_t max_height;        /* default 2048 */
  int32_t sorter_k;          /* per-pixel fixed-size sorter capacity K (the paper's "depth
                                filter", Sec. 2 "Sample blending", size 3): one of
                                1, 2, 3, 4, 6, 8, 12; default 3 */
  int32_t raster_ctas_per_sm;/* persistent rasteriser CTAs per SM; default: occupancy limit */
  int32_t ref_factor;        /* bin-reference capacity per quad in the workspace; default 4 */
  int32_t flags;             /* LR_FLAG_* */
  int32_t device;            /* CUDA device ordinal; -1 or 0 = current device */
  int32_t bin_size;          /* pixels per side of the binning stage's square bins: 16, 32 or
                                64 (Sec. 2, Stage 2 uses 32; Sec. 4 proposes 64 for sparse
                                and 16 for dense regions); default 32. Any bin size gives the
                                same exact image: it changes how many (quad, bin) references
                                binning makes and how large the per-bin depth sorts are. */
  int32_t block_h;           /* rows of the rasteriser's work item: 4 (8x4 half-blocks, the
                                default) or 8 (8x8 blocks, Sec. 2, Stage 3, Phase 2: a quad
                                meeting both halves is set up once). 8 applies to forward
                                exact renders with flat or per-vertex colours and sorter_k
                                1, 2 or 3; other renders of the context use 8x4. The image
                                is the same either way. */
  int32_t shared_setup;      /* 1: a CTA of 8 warps rasterises a 32x8 strip of a bin (one 8x4
                                half-block per warp) and sets each candidate triangle up once
                                for the strip in shared memory (Sec. 2, Stage 3: a bin's
                                workgroup sets up its triangles together); forward exact
                                renders with flat or per-vertex colours, sorter_k 1-3 and
                                32-pixel bins, the others as without it. 0 (default): every
                                warp sets up its half-block's candidates itself. */
} lr_config;

/* A quad scene (Sec. 2: quads, not triangles, are the input primitive). Device memory. */
typedef struct {
  const float* positions;    /* device f32[V][3], world space */
  int64_t num_vertices;      /* V */
  const uint32_t* indices;   /* device u32[Q][4] vertex indices, or NULL: quad q uses
                                vertices 4q..4q+3 (then V >= 4Q) */
  int64_t num_quads;         /* Q */
  const float* colors;       /* device, straight RGBA: f32[Q][4] (LR_COLOR_FLAT) or
                                f32[V][4] (LR_COLOR_VERTEX, interpolated perspective-correctly)
                                or f32[V][8] (LR_COLOR_LIT: RGBA, normal xyz, one unused
                                float; colour and normal interpolated perspective-correctly,
                                RGB then scaled by amb + (1 - amb) |n.L| / |n|, a two-sided
                                Lambert term plus ambient, alpha unchanged; not with
                                cov_hash or LR_FLAG_ALPHA_THRESHOLD: LR_ERR_UNSUPPORTED) */
  int32_t color_mode;
  int32_t reserved;
} lr_quads;

/* Camera: clip = view_proj * (x, y, z, 1), row-major; clip.w is the view depth (> 0 in
 * front). Quads with any vertex outside near_z <= w <= far_z are culled whole. */
typedef struct {
  float view_proj[16];
  float near_z, far_z;
} lr_camera;

/* Outputs of one view. rgba is required; the rest are optional (NULL). Device memory,
 * row 0 = top of the image. */
typedef struct {
  float* rgba;               /* f32[H][W][4]: composited straight RGB and coverage alpha */
  uint8_t* rgba8;            /* u8[H][W][4]: rint(clamp(v, 0, 1) * 255) */
  uint32_t* frag_count;      /* u32[H][W]: number of fragments covering the pixel */
  uint64_t* cov_hash;        /* u64[H][W]: sum of splitmix64(2 * quad + triangle) */
  uint32_t* exact_mask;      /* u32[ceil(H/4)][ceil(W/8)]: per 8x4 half-block, bit ly*8+lx set
                                if pixel (8 hx + lx, 4 hy + ly) took the exact (overflow) path;
                                lr_render_backward can take it to skip its own detection */
} lr_target;

/* One view of a batch: a scene, a camera, a resolution and its outputs.
 * owned_tiles: NULL (render the whole frame), or a device bit set over the frame's 32x32-
 * pixel tiles, u32[ceil(T / 32)] with T = ceil(W / 32) * ceil(H / 32) and tile
 * (tx, ty) = bit (ty * ceil(W / 32) + tx) % 32 of word (ty * ceil(W / 32) + tx) / 32.
 * With a set, setup and binning still process every quad of the scene, but only the owned
 * tiles are depth-sorted and rasterised, and only their pixels of every output (rgba,
 * rgba8, frag_count, cov_hash, exact_mask) are written; the rest of each output is left
 * as it was. This is the screen-space split of the sort-middle design (Sec. 2, "Pipeline
 * description": the screen is cut into bins that are rasterised independently): several
 * renderers can each take a disjoint tile set of one frame and the tiles are gathered
 * afterwards. lr_stats.fragments and overflow_pixels then count the owned tiles only.
 * Not with lr_render_backward's own view, lr_render_msaa or lr_render_noalloc (which take
 * no lr_view).
 * sorter_k: 0 (the context's sorter capacity) or the capacity for this view, one of 1, 2,
 * 3, 4, 6, 8, 12 (any capacity gives the same exact image; it only changes which pixels
 * take the exact path, and so the speed). All views of one lr_render_batch call must
 * resolve to the same capacity (LR_ERR_INVALID_ARG otherwise); the server batches only
 * requests of equal capacity. */
typedef struct {
  lr_quads quads;
  lr_camera camera;
  int32_t width, height;
  lr_target target;
  const uint32_t* owned_tiles;
  int32_t sorter_k;
  int32_t reserved;
} lr_view;

typedef struct {
  int32_t status;            /* sticky device-side status of the last render (lr_status) */
  int32_t n_views;
  int64_t quads_in;
  int64_t quads_visible;
  int64_t culled[8];         /* by reason: 1 bad index, 2 non-finite, 3 depth, 4 guard band,
                                5 degenerate, 6 no pixel centre */
  int64_t bin_refs;          /* (quad, bin) references produced by binning */
  int64_t bin_refs_capacity; /* what the workspace could hold */
  int64_t bins_nonempty;
  int64_t bins_high;         /* bins of 2048 or more references (sorted by the dense-bin path) */
  int64_t max_bin_refs;
  int64_t fragments;         /* covering (pixel, quad, triangle) fragments */
  int64_t overflow_pixels;   /* pixels re-done by the exact full sort */
  float stage_ms[8];         /* with LR_FLAG_TIMING: setup, count, scan, scatter, sort,
                                raster, overflow, total */
  int64_t sort_bins[3];      /* the bins_high bins by how their references were sorted:
                                [0] bucket sort in shared memory (up to 20480 references,
                                no bucket over 64), [1] merge sort in shared memory alone
                                (up to 8192), [2] merge sort of 8192-reference runs merged
                                through global memory (the rest) */
} lr_stats;

/* Byte offsets, inside a workspace, of the per-quad records written by the setup stage and
 * of the binning arrays (for tests and inspection; valid after the render's stream has
 * finished and until the workspace is reused):
 *   rec       u32[Q][16] per visible quad (not written for a culled one): X0 Y0 X1 Y1 X2
 *                        Y2 X3 Y3 (snapped, 1/256 pixel), the four vertices' 1/w (f32 bits),
 *                        1/|A0| and 1/|A1| (f32 bits of the reciprocal doubled triangle
 *                        areas, 0 for a zero-area triangle), info (as rec_info, cull reason
 *                        0), 0
 *   rec_rect  u32[Q][2]  pixel-centre AABB: px0 | px1 << 16, py0 | py1 << 16
 *                        (0x0000FFFF, 0x0000FFFF for a culled quad)
 *   rec_info  u32[Q]     bit 0/1: triangle 0/1 has non-zero area, bit 2: spans more than
 *                        4x4 bins, bit 3: all vertices at the same 1/w, bits 4/5: triangle
 *                        0/1 has negative area (v1, v2 swapped), bits 6/7: triangle 0/1 is
 *                        small enough for 32-bit edge arithmetic, bits 8..11: cull reason
 *                        (0 = visible)
 *   bin_off   u32[bins+1] start of each bin's reference list in refs
 *   refs      u64[capacity] per-bin reference lists, sorted front to back
 * Quads, bins and pixels of a batch are numbered view after view. */
typedef struct {
  size_t rec, rec_rect, rec_info, bin_count, bin_off, refs;
  int64_t total_quads, total_bins, refs_capacity;
} lr_ws_layout;

/* Create / destroy a context bound to one CUDA device. */
lr_status lr_create(const lr_config* config, lr_ctx** out_ctx);

/* Light of LR_COLOR_LIT views rendered on this context from now on (also by graphs
 * created later and by a server started later). light_dir: host float[3], the direction
 * toward the light in world space (any non-zero length; normalised here); ambient in
 * [0, 1]. Default: direction (0, 0, 1), ambient 0.25. LR_ERR_INVALID_ARG for a zero or
 * non-finite direction or an ambient outside [0, 1]. */
lr_status lr_set_lighting(lr_ctx* ctx, const float* light_dir, float ambient);
lr_status lr_destroy(lr_ctx* ctx);

/* Bytes of workspace lr_render needs for a scene of num_quads quads at width x height
 * (host call, no GPU work). The workspace holds fixed-size arrays plus the (quad, bin)
 * reference lists of binning, whose capacity is whatever the workspace holds beyond the
 * fixed part; this function sizes it at ref_factor references per quad. A scene whose
 * quads overlap more bins reports LR_ERR_OVERFLOW from lr_get_stats, with stats.bin_refs
 * = the number of references it needed; lr_workspace_size_refs gives the bytes for that. */
lr_status lr_workspace_size(const lr_ctx* ctx, int64_t num_quads, int32_t width, int32_t height,
                            size_t* out_bytes);

/* Same for a batch of views (host memory array of n_views lr_view). */
lr_status lr_workspace_size_batch(const lr_ctx* ctx, int32_t n_views, const lr_view* views,
                                  size_t* out_bytes);

/* Bytes of workspace for a batch whose binning produces bin_refs references (-1: the
 * default capacity of ref_factor per quad). */
lr_status lr_workspace_size_refs(const lr_ctx* ctx, int32_t n_views, const lr_view* views,
                                 int64_t bin_refs, size_t* out_bytes);

/* Render one frame (Sec. 2, all three stages): out_rgba = device f32[H][W][4].
 * workspace: device, >= lr_workspace_size bytes, 256-byte aligned, owned by the caller.
 * Enqueued on stream; returns LR_ERR_INVALID_ARG / LR_ERR_TOO_LARGE / LR_ERR_OOM for bad
 * arguments before any GPU work. */
lr_status lr_render(lr_ctx* ctx, const lr_quads* quads, const lr_camera* camera, int32_t width,
                    int32_t height, float* out_rgba, void* workspace, size_t workspace_bytes,
                    lr_stream stream);

/* Render n_views views (host array) with one launch per pipeline stage: every stage's
 * kernel processes all views' quads, bins and pixels together (persistent multi-view
 * launch). The launch sequence contains no host synchronisation, so it can be captured
 * in a CUDA graph. */
lr_status lr_render_batch(lr_ctx* ctx, int32_t n_views, const lr_view* views, void* workspace,
                          size_t workspace_bytes, lr_stream stream);

/* ---- captured batches -------------------------------------------------------------
 * lr_graph_create captures the launch sequence of lr_render_batch for these views into a
 * CUDA graph bound to this workspace. lr_graph_launch replays it on a stream; views may
 * be NULL (render the captured views again) or new views with the same shapes (per view:
 * width, height, num_quads, color_mode, whether a coverage hash is written, sorter
 * capacity); scene and output pointers, owned-tile sets and cameras may change.
 * Replays read the view descriptors from one of two pinned host buffers owned by the
 * graph; a launch waits (host side) for the replay two launches back. The graph, its
 * workspace and the context must outlive every replay; lr_get_stats reports the last one. */
typedef struct lr_graph lr_graph;
lr_status lr_graph_create(lr_ctx* ctx, int32_t n_views, const lr_view* views, void* workspace,
                          size_t workspace_bytes, lr_graph** out_graph);
lr_status lr_graph_launch(lr_graph* graph, const lr_view* views, lr_stream stream);
lr_status lr_graph_destroy(lr_graph* graph);

/* Backward pass of the compositing with respect to flat per-quad RGBA.
 * grad_out: device f32[H][W][4] = dL/d(R, G, B, A) of the rendered image.
 * fwd_rgba: device f32[H][W][4] = the forward image of the same scene (as lr_render wrote
 *           it); the per-pixel fragment order is recomputed, not stored.
 * exact_mask: NULL, or the forward's lr_target.exact_mask for this scene rendered on a
 *           context with the same sorter capacity. Without it the rasteriser streams every
 *           half-block twice (first to find the pixels the fixed-size sorter cannot order,
 *           which take the exact path, then with gradients); with it, once. A pixel the
 *           mask misses makes lr_get_stats report LR_ERR_MASK_MISMATCH, and the gradients
 *           of that call are not valid (call again without the mask).
 * grad_colors: device f32[Q][4]; gradients are ADDED to it (zero it first).
 * Only LR_COLOR_FLAT scenes (LR_ERR_UNSUPPORTED otherwise). */
lr_status lr_render_backward(lr_ctx* ctx, const lr_quads* quads, const lr_camera* camera,
                             int32_t width, int32_t height, const float* fwd_rgba,
                             const float* grad_out, const uint32_t* exact_mask, float* grad_colors,
                             void* workspace, size_t workspace_bytes, lr_stream stream);

/* Layout of a workspace of workspace_bytes bytes for this batch (host call). */
lr_status lr_workspace_layout(const lr_ctx* ctx, int32_t n_views, const lr_view* views,
                              size_t workspace_bytes, lr_ws_layout* out);

/* Wait for the last render / backward issued on this context and report its counters
 * (synchronises that stream). stats may be NULL to only fetch the status. */
lr_status lr_get_stats(lr_ctx* ctx, lr_stats* stats);

/* Human-readable description of the last error on this context (never NULL). */
const char* lr_last_error(const lr_ctx* ctx);

/* ---- rendering without any allocation -------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory when they render: for example a plugin that a host application
 * calls once per frame, where the host owns all device memory through its own pool and
 * forbids cudaMalloc after start-up (an allocation there can stall every stream of the
 * process and may not fit the host's memory budget), so such a caller also cannot provide
 * the workspace lr_render needs.
 *
 * lr_render_noalloc renders one frame like lr_render with the default sorter capacity
 * (K = 3), but uses as its workspace a device array of LR_NOALLOC_SCRATCH_BYTES bytes that
 * is part of the library's device code (every GPU on which that code is loaded holds it
 * until the process exits). It needs no lr_ctx and calls no allocating function (no
 * cudaMalloc / cudaFree / cudaMallocHost, no host heap).
 *  - quads, camera: as for lr_render (device scene, host camera struct), with flat or
 *    per-vertex colours (LR_COLOR_LIT scenes: LR_ERR_INVALID_ARG).
 *  - out_rgba: device f32[H][W][4], 16-byte aligned; written when the stream reaches it.
 *  - device_status: NULL, or a device int32 that receives the GPU-side status of this call
 *    (LR_OK, LR_ERR_OVERFLOW if the scene's bin references did not fit the array,
 *    LR_ERR_INVALID_ARG for out-of-range vertex indices); read it after the stream syncs.
 *    The host-side size check below guarantees room for two references per quad only; a
 *    scene of larger quads can still need more, and then the GPU reports LR_ERR_OVERFLOW
 *    and leaves out_rgba unwritten. With device_status NULL nothing reports that case, so
 *    a caller that cannot rule it out should pass a status word.
 *  - Returns LR_ERR_TOO_LARGE, before any GPU work, when the scene's records plus at least
 *    two bin references per quad do not fit in LR_NOALLOC_SCRATCH_BYTES (roughly: up to
 *    about 480k quads at 1920x1080, or 550k quads at 256x256); LR_ERR_INVALID_ARG for bad
 *    arguments; LR_ERR_CUDA if a launch or the set-up failed.
 *  - The first call on each device (with that device current) looks up the array's
 *    address and sets kernel attributes; make that first call before any stream capture.
 *  - All calls share the array, which keeps the last call's contents; each call zeroes
 *    what must start at zero. Calls whose GPU work overlaps (e.g. on two streams) race on
 *    the array: serialise them. */
#define LR_NOALLOC_SCRATCH_BYTES (64ull << 20)
lr_status lr_render_noalloc(const lr_quads* quads, const lr_camera* camera, int32_t width,
                            int32_t height, float* out_rgba, int32_t* device_status,
                            lr_stream stream);

/* ---- multisampling ------------------------------------------------------------------
 * (The paper's prototype has no anti-aliasing; Sec. 4, "Future work", names 4x and 16x
 * multisample anti-aliasing as an extension that mainly changes the coverage and blending
 * phases of the raster stage.) lr_render_msaa renders one frame with n_samples sample
 * positions per pixel. Every sample gets the exact composite of the fragments covering it
 * (coverage, depth key and colour taken at the sample, same order and tie rule as
 * lr_render); the output pixel is the mean of its samples (fp32 sum in sample order,
 * divided by n_samples). The samples are the views of one batched render (every stage
 * launched once for all samples), followed by one resolve kernel.
 *  - quads, camera: as for lr_render.
 *  - n_samples: 1..16.
 *  - sample_offsets: host int32[n_samples][2], the offsets (dx, dy) of the samples from the
 *    pixel centre in 1/256 px (x right, y down), each in [-127, 127]; or NULL for the default
 *    pattern of n_samples = 4 (a rotated grid: offsets (+-1/8, +-3/8) px, one sample per row
 *    and column of a 4x4 sub-grid) or 16 (one sample per row and column of a 16x16 sub-grid,
 *    row i, counted from the top, in column (5 i + 3) mod 16).
 *  - out_rgba: device f32[H][W][4], 16-byte aligned.
 *  - workspace: device, 256-byte aligned, at least lr_workspace_size_msaa() bytes: the
 *    per-sample images (16 B per pixel and sample) followed by the batch's workspace.
 *  - Returns LR_ERR_INVALID_ARG for n_samples outside 1..16, NULL offsets with n_samples
 *    other than 4 or 16, an offset outside [-127, 127] or bad pointers; LR_ERR_OOM when the
 *    workspace is too small; otherwise as lr_render. lr_get_stats reports the samples as
 *    views (fragments summed over the samples). */
lr_status lr_workspace_size_msaa(const lr_ctx* ctx, int64_t num_quads, int32_t width, int32_t height,
                                 int32_t n_samples, size_t* out_bytes);
lr_status lr_render_msaa(lr_ctx* ctx, const lr_quads* quads, const lr_camera* camera, int32_t width,
                         int32_t height, int32_t n_samples, const int32_t* sample_offsets, float* out_rgba,
                         void* workspace, size_t workspace_bytes, lr_stream stream);

/* ---- serving: continuous batching of render requests ------------------------------
 * (Not in the paper; it serves the single-frame pipeline.) A host thread keeps
 * num_slots batches in flight, each on its own CUDA stream with its own device workspace
 * of slot_workspace_bytes (allocated by lr_server_start, freed by lr_server_stop or
 * lr_destroy). Queued requests are admitted in arrival order into the next free slot
 * while the batch fits the slot's workspace and has at most max_batch_views views; each
 * batch is one multi-view render (lr_render_batch). A request whose view does not fit a
 * slot alone completes with LR_ERR_OOM. While a server runs on a context, call only
 * lr_submit / lr_poll / lr_poll_info / lr_server_get_stats / lr_server_stop on it (these
 * may be called from any thread). */
typedef struct {
  int32_t num_slots;             /* batches in flight at once; default 2 */
  int32_t max_batch_views;       /* views per batch; default 16 */
  int64_t slot_workspace_bytes;  /* device workspace per slot; default 512 MiB */
  int32_t poll_interval_us;      /* while batches run, the server thread polls their completion
                                    in a spin for up to this long between looks at the queue
                                    (new requests end the spin early); default 20 */
  int32_t idle_spin_us;          /* with nothing queued or running, the server thread spins this
                                    long waiting for a request before it sleeps (waking a
                                    sleeping thread costs tens of microseconds of latency; the
                                    spin costs one CPU core); 0 = default 5000, -1 = sleep at
                                    once */
} lr_server_config;

typedef struct {
  uint64_t submit_ns, launch_ns, done_ns;   /* lr_now_ns() clock */
  int32_t batch_views;                      /* views in the batch that rendered it */
  int32_t reserved;
} lr_request_info;

typedef struct {
  int64_t submitted, completed, failed, batches, batched_views, split_batches, queued;
} lr_server_stats;

lr_status lr_server_start(lr_ctx* ctx, const lr_server_config* config);
/* Finishes every queued and running request, then stops the thread and frees the slots. */
lr_status lr_server_stop(lr_ctx* ctx);
/* Queue a render request. view (host struct) holds device pointers to the scene and the
 * outputs, which the caller keeps alive and unmodified until lr_poll reports completion.
 * Arguments are checked as lr_render_batch checks them; a bad request is refused here
 * (LR_ERR_INVALID_ARG / LR_ERR_TOO_LARGE) and never joins a batch. */
lr_status lr_submit(lr_ctx* ctx, const lr_view* view, uint64_t* ticket);
/* Completion of a ticket, waiting at most timeout_us microseconds. Returns LR_OK with
 * *result = the request's status once it has finished (the ticket is then released),
 * LR_PENDING (timeout_us == 0) or LR_ERR_TIMEOUT (timeout_us > 0) if it has not. */
lr_status lr_poll(lr_ctx* ctx, uint64_t ticket, int32_t timeout_us, lr_status* result);
/* lr_poll plus the request's submit / launch / completion times and batch size. */
lr_status lr_poll_info(lr_ctx* ctx, uint64_t ticket, int32_t timeout_us, lr_status* result,
                       lr_request_info* info);
lr_status lr_server_get_stats(lr_ctx* ctx, lr_server_stats* stats);
/* The monotonic clock (nanoseconds) used for lr_request_info. */
uint64_t lr_now_ns(void);

#ifdef __cplusplus
}
#endif

#endif /* LR_H_ */
