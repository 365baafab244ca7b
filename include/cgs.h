/*
 * cgs.h -- C ABI of libcgs.so, a B300 (sm_103a) implementation of the rendering hot path
 * of CityGaussian (arXiv 2404.01133): block-wise level-of-detail selection over a
 * block-partitioned Gaussian scene (Sec. 3.3.2), followed by 3D Gaussian Splatting tile
 * rasterization (Eq. 1, Sec. 3.1) and its analytic backward pass.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named d_* (and every pointer inside cgs_scene and cgs_frame) are DEVICE
 *    pointers owned by the caller.  No entry point of this header allocates or frees
 *    device memory or keeps a pointer after it returns.
 *  - Every call only enqueues work on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and returns; only cgs_frame_status synchronizes.  A forward runs its long-tile
 *    sort on a side stream that the library keeps per host thread and device, forked from
 *    `stream` after the entries are binned and joined back into it before compositing: the
 *    work still starts after everything enqueued on `stream` before the call and ends before
 *    anything enqueued after it, also under stream capture.
 *  - The return value is CGS_OK or the code of a failed host-side argument check or
 *    launch.  Conditions found on the device (capacity overflow, a bounded inter-block
 *    wait that gave up) are latched in the frame's device status word and reported by
 *    cgs_frame_status.  No entry point aborts, traps or waits without bound.
 *  - Floating-point inputs are FP32.  Gaussian attributes are ACTIVATED values: linear
 *    scales, opacity in (0, 1), rotation quaternion (w, x, y, z) of any length
 *    (normalised inside, Hamilton convention).
 *  - Cameras use OpenCV axes (x right, y down, z forward), x_cam = R x_world + t; pixel
 *    (i, j) has its centre at the integer coordinate (i, j).
 */
#ifndef CGS_H
#define CGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CGS_OK 0
#define CGS_ERR_INVALID_ARGUMENT 1
#define CGS_ERR_WORKSPACE_TOO_SMALL 2
#define CGS_ERR_CAPACITY 3     /* device: more selected Gaussians or tile entries than the frame holds */
#define CGS_ERR_SPIN_TIMEOUT 4 /* device: a bounded inter-block wait gave up; outputs are invalid */
#define CGS_ERR_CUDA 5         /* a CUDA launch or memset failed */
#define CGS_ERR_UNSUPPORTED 6
#define CGS_ERR_TOO_LARGE 7    /* request exceeds the fixed limits of cgs_render_forward_static */

/* Pinhole camera of one view: intrinsics kappa and pose tau_i of Eq. 1 (Sec. 3.1). 96 bytes. */
typedef struct cgs_camera {
    float R[9];        /* world -> camera rotation, row major */
    float t[3];        /* world -> camera translation */
    float campos[3];   /* camera centre in world coordinates (= -R^T t) */
    float fx, fy, cx, cy;
    int32_t width, height;
    float _pad[3];
} cgs_camera;

/* Block-partitioned Gaussian scene.  Per Gaussian (Sec. 3.1): position, opacity, scale and
 * rotation (the covariance), SH features.  With attr_fp16 the non-position attributes are
 * stored in half precision (the transfer variant noted, commented out, after Sec. 3.3.2:
 * position FP32, the other properties FP16; opacity stays with the position here).
 * SH features are in R^{3x16} at degree 3.  Detail level l of block
 * b (Sec. 3.3.1/3.3.2) is the index range [level_offset[b*L + l], + level_count[b*L + l]).
 * Level 0 is the finest.  Segments of different blocks must not overlap and must ascend
 * with b, because scene index order breaks depth ties.  A scene without blocks is one
 * block with one level covering [0, n). */
typedef struct cgs_scene {
    const float* mean_opac;      /* [n][4] x, y, z, opacity */
    const float* scale;          /* [n][4] sx, sy, sz, unused */
    const float* quat;           /* [n][4] w, x, y, z */
    const float* sh;             /* [n][(sh_degree+1)^2][3] SH coefficients, channel fastest */
    int64_t n;                   /* Gaussians, < 2^31 */
    int32_t sh_degree;           /* 0..3 */
    int32_t n_blocks;            /* 1 .. 2^20 - 1 */
    int32_t n_levels;            /* >= 1 */
    int32_t attr_fp16;           /* 0: scale, quat, sh are FP32 as above; 1: they are IEEE half
                                    (binary16) with the same shapes ([n][4], [n][4],
                                    [n][(deg+1)^2][3]); mean_opac stays FP32.  Gradients are FP32
                                    in the FP32 layout either way. */
    const int64_t* level_offset; /* [n_blocks][n_levels] */
    const int64_t* level_count;  /* [n_blocks][n_levels] */
    const float* block_aabb;     /* [n_blocks][6] lo xyz, hi xyz: Eq. 7 bounds (cgs_block_bounds) */
    const float* block_cell;     /* [n_blocks][4] x0, x1, y0, y1 ground cell of the block */
} cgs_scene;

/* Rendering parameters. */
typedef struct cgs_config {
    int32_t tile;        /* tile side in pixels: 16 or 8 */
    int32_t batch;       /* Gaussians staged per round by the compositing kernels: 32..256, a
                            multiple of 32 and at most tile*tile */
    float near_z;        /* near plane on camera-space z (0.2) */
    float bg[3];         /* background colour */
    double lod_dist[2];  /* level thresholds d1 < d2 in scene units: level 0 if dmin < d1,
                            1 if dmin < d2, else 2 */
    int32_t lod_mode;    /* when the renderer selects levels itself (no d_levels, no
                            d_view_block): CGS_LOD_BLOCK or CGS_LOD_POINT */
    int32_t exact;       /* 0: the fast compositing path.  1: the parity build of the
                            compositing kernels (forward and backward): each pair's power,
                            falloff and alpha in the operations and order of Eq. 1's plain
                            per-pixel loop, e^power rounded once to FP32 from the FP64
                            exponential, transmittance T (1 - alpha) and colour C + c alpha T
                            with two roundings each; slow (one FP64 exponential per pair),
                            for parity checks.  Not available for cgs_render_forward_hits
                            (CGS_ERR_UNSUPPORTED). */
} cgs_config;

/* Level selection modes.
 * CGS_LOD_BLOCK: the paper's block-wise selection (Sec. 3.3.2, cgs_lod_select).
 * CGS_LOD_POINT: the point-wise baseline the paper compares against (Sec. 3.3.2; Table 5, the LoD-strategy ablation):
 *   every non-empty block takes part without block culling; a Gaussian of block b at rank r
 *   in the block's finest level (levels are nested prefixes) is rendered iff
 *   r < level_count[b][l], l = 0 if dist < d1, 1 if dist < d2, else 2 (clamped), with
 *   dist = sqrt((dx*dx + dy*dy) + dz*dz) in FP32 from the camera centre to its mean. */
#define CGS_LOD_BLOCK 0
#define CGS_LOD_POINT 1

/* A batch of n_views equally sized views rendered together, and the caller-owned device
 * workspace holding its intermediate state (kept for the backward).  n_cap bounds the
 * selected Gaussians summed over the views (< 2^31); k_cap bounds the (tile, Gaussian)
 * entries summed over the views (< 2^30).  Size ws with cgs_frame_workspace_bytes and fill
 * it with zeros once, before its first use: the backward's per-Gaussian accumulators are
 * kept at zero between backwards by the library (each backward clears what it added), not
 * cleared by every forward.  flags: 0, or CGS_FRAME_NO_PAIR_COUNT. */
typedef struct cgs_frame {
    void* ws;
    int64_t ws_bytes;
    int32_t n_views, width, height, tile, n_blocks;
    int32_t flags;
    int64_t n_cap;
    int64_t k_cap;
} cgs_frame;

/* cgs_frame.flags: the compositing backward does not count the contributing (pixel,
 * Gaussian) pairs it replays (cgs_frame_status counts[4] stays 0).  The count is a diagnostic
 * (it sizes the algorithmic work of a roofline and checks that the backward replays the
 * forward's blends); leaving it out saves a few instructions per replayed entry and changes
 * no other output. */
#define CGS_FRAME_NO_PAIR_COUNT 1

int32_t cgs_version(void);
const char* cgs_status_string(int32_t code);

/* Bytes of workspace a cgs_frame with these dimensions needs; 0 if they are invalid. */
int64_t cgs_frame_workspace_bytes(int32_t n_views, int32_t width, int32_t height, int32_t tile,
                                  int32_t n_blocks, int64_t n_cap, int64_t k_cap);

/* Eq. 7 (Sec. 3.3.2), per block and axis over the means of the block's finest level:
 *   MAD = median(|p - median(p)|),
 *   lo = max(min p, median - n_mad MAD),  hi = min(max p, median + n_mad MAD),
 * evaluated in FP64 (median of an even count = mean of the two middle values), stored in
 * d_aabb [n_blocks][6] rounded outward to FP32.  Exact selection, deterministic.  d_ws
 * holds cgs_block_bounds_workspace_bytes(scene->n) bytes. */
int64_t cgs_block_bounds_workspace_bytes(int64_t n);
int32_t cgs_block_bounds(const cgs_scene* scene, double n_mad, float* d_aabb, void* d_ws, int64_t ws_bytes,
                         void* stream);

/* ---- Scene upload (Sec. 3.1 attributes, Sec. 3.3.2 per-block detail levels) --------------
 * The library keeps no scene of its own: a cgs_scene describes caller-owned device arrays.
 * cgs_scene_upload fills one from host arrays in ONE caller-owned device buffer of
 * cgs_scene_bytes(...) bytes (d_mem, 256-byte aligned, which the caller frees after the last
 * call that uses the scene): it copies the attributes (layouts as in cgs_scene; scale, quat
 * and sh in IEEE half when attr_fp16 = 1), the block table level_offset / level_count
 * [n_blocks][n_levels] and block_cell [n_blocks][4] with one cudaMemcpyAsync each on `stream`
 * (pageable host memory makes those copies wait for the host), then, for n_mad >= 0, writes
 * the Eq. 7 block bounds (cgs_block_bounds); for n_mad < 0 the bounds are zero (scenes
 * rendered with explicit levels or per-view blocks need none).  *out receives the descriptor.
 * The block table is checked on the host first: every segment within [0, n), and the
 * blocks' segments ascending and not overlapping (scene order breaks depth ties); a
 * violation, a null pointer or an invalid size returns CGS_ERR_INVALID_ARGUMENT, a short
 * buffer CGS_ERR_WORKSPACE_TOO_SMALL, both before any device work.  cgs_scene_bytes returns
 * -1 for invalid sizes. */
int64_t cgs_scene_bytes(int64_t n, int32_t sh_degree, int32_t n_blocks, int32_t n_levels, int32_t attr_fp16);
int32_t cgs_scene_upload(cgs_scene* out, void* d_mem, int64_t mem_bytes, const float* h_mean_opac,
                         const void* h_scale, const void* h_quat, const void* h_sh, int64_t n, int32_t sh_degree,
                         int32_t attr_fp16, int32_t n_blocks, int32_t n_levels, const int64_t* h_level_offset,
                         const int64_t* h_level_count, const float* h_block_cell, double n_mad, void* stream);

/* Block-wise level selection and frustum culling (Sec. 3.3.2) in FP64 for n_views
 * cameras: the corners of a block's box with camera-space z > near_z are projected; the
 * block is visible if their screen bounding box overlaps the image (x in (-0.5, W-0.5),
 * y in (-0.5, H-0.5)); the block whose ground cell holds the camera is always kept; the
 * level follows the minimum distance from the 8 corners to the camera centre.  Writes
 * d_levels [n_views][n_blocks]: -1 culled or empty, else the level (<= n_levels - 1). */
int32_t cgs_lod_select(const cgs_scene* scene, const cgs_config* cfg, const cgs_camera* d_cams,
                       int32_t n_views, int8_t* d_levels, void* stream);

/* Forward render of the frame's views (Eq. 1, Sec. 3.1) over the selected Gaussians,
 * fused by concatenation (Sec. 3.2.3, 3.3.2).  Per view v the rendered set is:
 *   d_levels != NULL:     segments (b, d_levels[v*n_blocks + b]) with a level >= 0;
 *   d_view_block != NULL: block d_view_block[v] at level 0 (per-block training views);
 *   both NULL:            the cgs_lod_select choice for d_cams[v].
 * d_cams holds n_views cameras of size frame->width x frame->height.  Writes d_image
 * [n_views][3][H][W], d_final_T [n_views][H][W] and d_n_contrib [n_views][H][W] (one past
 * the position, in the pixel's tile list, of its last blended Gaussian) and keeps the
 * sorted per-tile lists in frame->ws for cgs_render_backward. */
int32_t cgs_render_forward(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                           const cgs_camera* d_cams, const int32_t* d_view_block, const int8_t* d_levels,
                           float* d_image, float* d_final_T, uint32_t* d_n_contrib, void* stream);

/* Analytic backward of cgs_render_forward (differentiable rendering, Sec. 3.1) for the
 * same scene, frame, config and cameras, replaying every pixel back to front from its
 * final transmittance and n_contrib.  ADDS dL/d(attribute) into gradient buffers laid out
 * like the scene: d_g_mean_opac [n][4] (x, y, z, opacity), d_g_scale [n][4], d_g_quat
 * [n][4], d_g_sh [n][(deg+1)^2][3].  Discrete decisions (culls, clamps, skips, the stop)
 * pass no gradient.  Accumulation order is not fixed: repeated runs may differ in the
 * last bits. */
int32_t cgs_render_backward(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                            const cgs_camera* d_cams, const float* d_dL_dimage, const float* d_final_T,
                            const uint32_t* d_n_contrib, float* d_g_mean_opac, float* d_g_scale,
                            float* d_g_quat, float* d_g_sh, void* stream);

/* The same backward with the gradients of each visible (view, Gaussian) pair in its own
 * row instead of added into scene-indexed arrays.  Rows r = 0 .. n_vis-1 (n_vis: the
 * visible count of the frame, cgs_frame_status counts[1]) are WRITTEN, in the order of the
 * visible list (frame buffer 7): d_g_mean_opac [rows][4] (x, y, z, opacity), d_g_scale
 * [rows][4] (x, y, z, 0), d_g_quat [rows][4], d_g_sh [rows][(deg+1)^2][3] and d_g_index
 * [rows] (int64 scene index of the row's Gaussian).  Arrays hold frame->n_cap rows; rows
 * from n_vis on are left as they are.  Nothing needs clearing between calls, and with one
 * view per frame every scene index appears at most once; with several views the caller
 * sums rows of equal index.  Results equal cgs_render_backward's up to the order of
 * floating-point additions. */
int32_t cgs_render_backward_packed(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                                   const cgs_camera* d_cams, const float* d_dL_dimage, const float* d_final_T,
                                   const uint32_t* d_n_contrib, float* d_g_mean_opac, float* d_g_scale,
                                   float* d_g_quat, float* d_g_sh, int64_t* d_g_index, void* stream);

/* The L1 loss and the backward in one pass (Sec. 3.2.3's L1 term, Sec. 3.1's differentiable
 * rendering): equivalent to cgs_l1_loss (target_u8 = 0: d_target is float) or cgs_l1_loss_u8
 * (target_u8 = 1: d_target is uint8_t, t standing for t / 255) over the frame's whole image,
 * count = n_views * 3 * height * width, followed by cgs_render_backward (d_g_index = NULL:
 * gradients ADDED into scene-indexed arrays) or cgs_render_backward_packed (d_g_index != NULL:
 * rows WRITTEN), without the gradient image: the compositing backward forms each pixel's
 * dL/dimage = sign(img - target) / count from d_image (the forward's output, [n_views][3][H][W])
 * and d_target (same layout) where it reads it.  ADDS mean |img - target| into *d_loss (atomic
 * adds, so the summation order is not fixed).  The per-pixel gradient equals cgs_l1_loss's bit
 * for bit.  CGS_ERR_UNSUPPORTED for the parity configuration (cfg->exact); other errors as
 * cgs_render_backward. */
int32_t cgs_render_backward_l1(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                               const cgs_camera* d_cams, const float* d_image, const void* d_target,
                               int32_t target_u8, const float* d_final_T, const uint32_t* d_n_contrib,
                               float* d_loss, float* d_g_mean_opac, float* d_g_scale, float* d_g_quat,
                               float* d_g_sh, int64_t* d_g_index, void* stream);

/* L1 photometric loss (the L1 term of the training loss, Sec. 3.2.3) over `count` values:
 * ADDS mean|img - target| into *d_loss and writes d_grad = sign(img - target) / count
 * (sign(0) = 0). */
int32_t cgs_l1_loss(const float* d_img, const float* d_target, int64_t count, float* d_loss, float* d_grad,
                    void* stream);

/* cgs_l1_loss with an 8-bit target (training images as decoded: channel value t stands for
 * t / 255, the FP32 quotient correctly rounded), same layout and outputs.  A quarter of the
 * target bytes of the FP32 variant. */
int32_t cgs_l1_loss_u8(const float* d_img, const uint8_t* d_target, int64_t count, float* d_loss, float* d_grad,
                       void* stream);

/* Synchronizes `stream`, then copies the frame's device status word to *status and its
 * counters to counts[0..7]: selected Gaussians, visible Gaussians, tile entries, forward
 * evaluated pairs (entries walked per pixel up to its stop), backward contributing pairs,
 * bounded-wait give-ups, forward (warp, entry) steps visited after culling, and steps in
 * which the entry blended into a pixel of the warp.  Either output may be NULL.  Returns
 * the status word (CGS_OK when nothing was latched). */
int32_t cgs_frame_status(const cgs_frame* frame, int32_t* status, int64_t* counts, void* stream);

/* Forward render of ONE view with no caller workspace and no allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc or hold a
 * workspace -- an application that owns all device memory and forbids allocation inside its
 * frame loop, or a plugin handed only its input and output buffers.  Same inputs, outputs
 * and results as cgs_render_forward for a one-view frame; the intermediate state lives in a
 * fixed device array of CGS_STATIC_WORKSPACE_BYTES inside the library, which every GPU that
 * loads the library keeps until the process exits.
 *  - Limits: width * height <= CGS_STATIC_MAX_PIXELS, scene->n <= CGS_STATIC_MAX_GAUSSIANS,
 *    scene->n_blocks <= CGS_STATIC_MAX_BLOCKS; larger requests return CGS_ERR_TOO_LARGE
 *    before any device work.  More than CGS_STATIC_MAX_ENTRIES (tile, Gaussian) entries sets
 *    CGS_ERR_CAPACITY in the device status.
 *  - d_status (device int32, may be NULL) receives the device status of this call as a CGS_*
 *    code, written on `stream` after the render.
 *  - Every call looks up the array's device address on the current device (the first lookup
 *    on a device loads the library there); make the first call on a device before any stream
 *    capture.  Nothing is cached, so calls after a cudaDeviceReset find the array again.
 *  - Every call uses the same array and clears what must start at zero; calls that overlap
 *    on the GPU (other streams, other host threads) race and must be serialized by the
 *    caller.  d_image etc. stay valid after later calls; the array's contents do not. */
#define CGS_STATIC_MAX_PIXELS (256 * 256)
#define CGS_STATIC_MAX_GAUSSIANS 32768
#define CGS_STATIC_MAX_ENTRIES 262144
#define CGS_STATIC_MAX_BLOCKS 64
#define CGS_STATIC_WORKSPACE_BYTES (12 << 20)
int32_t cgs_render_forward_static(const cgs_scene* scene, const cgs_config* cfg, const cgs_camera* d_cam,
                                  int32_t width, int32_t height, const int32_t* d_view_block,
                                  const int8_t* d_levels, float* d_image, float* d_final_T,
                                  uint32_t* d_n_contrib, int32_t* d_status, void* stream);

/* ---- Autotuner ------------------------------------------------------------------------------
 * Picks the tile size and the compositing batch depth of cgs_config for a workload by timing
 * the real step on the device: for each candidate (tile, batch) in the order
 *   (16, 256) (16, 128) (16, 64) (16, 32) (8, 64) (8, 32)
 * one warm-up call and `reps` timed calls (CUDA events on `stream`, median) of
 * cgs_render_forward (mode CGS_TUNE_FORWARD) or cgs_render_forward + cgs_render_backward_packed
 * with an upstream gradient of 1/(3 n_views W H) on every pixel (CGS_TUNE_FORWARD_BACKWARD),
 * over the given scene, cameras, selection (d_view_block / d_levels as in cgs_render_forward)
 * and frame capacities.  A candidate whose frame reports a device error (a capacity too small
 * for its tile size) is not eligible.  Writes the fastest choice into inout->tile and
 * inout->batch (the other fields of *inout are used as given) and, if ms_out is not NULL, the
 * candidates' median milliseconds into ms_out[CGS_TUNE_CANDIDATES] (-1: not eligible).
 * d_ws holds cgs_autotune_workspace_bytes(...) bytes of device memory (frames, outputs and
 * gradient rows of the candidates; its contents are overwritten).  Synchronises `stream`.
 * With cache_path, a text file of lines "<device name>|<cache_key> <tile> <batch>" is read
 * first (a hit returns at once, ms_out left at -1) and the choice appended to it.  Returns
 * CGS_ERR_CAPACITY when no candidate fits, CGS_ERR_INVALID_ARGUMENT for invalid arguments.
 * cgs_autotune_workspace_bytes returns -1 for invalid sizes. */
#define CGS_TUNE_CANDIDATES 6
#define CGS_TUNE_FORWARD 0
#define CGS_TUNE_FORWARD_BACKWARD 1
int64_t cgs_autotune_workspace_bytes(int32_t n_views, int32_t width, int32_t height, int32_t n_blocks, int64_t n_cap,
                                     int64_t k_cap, int32_t sh_degree, int32_t mode);
int32_t cgs_autotune(const cgs_scene* scene, const cgs_camera* d_cams, int32_t n_views, int32_t width, int32_t height,
                     const int32_t* d_view_block, const int8_t* d_levels, int64_t n_cap, int64_t k_cap, int32_t mode,
                     int32_t reps, void* d_ws, int64_t ws_bytes, cgs_config* inout, float* ms_out,
                     const char* cache_path, const char* cache_key, void* stream);

/* Device address and capacity (elements) of an internal frame array, valid after
 * cgs_render_forward; for parity tests and debugging.  which:
 *   0 sorted tile keys    u32 [k_cap]  view * tiles_per_view + tile (row-major tile id)
 *   1 sorted values       u32 [k_cap]  selected index (position in the concatenation)
 *   2 tile ranges         u32 [n_views * tiles][2]  [start, end) into 0/1
 *   3 scene index         u32 [n_cap]  selected index -> scene index
 *   4 projected records   float [n_cap][12]  u, v, opacity, ext_x | A', B', C', ext_y |
 *                                            r, g, b, view (ext: half-extent of alpha >= 1/255)
 *   5 tiles touched       u32 [n_cap]
 *   6 selected per view   u32 [n_views + 1] exclusive prefix of the per-view counts
 *   7 visible list        u32 [n_cap]  selected indices of the visible Gaussians (no fixed order)
 *   8 depth keys          u64 [n_cap]  view << 32 | FP32 depth bits (visible entries only)
 *   9 tile rects          u32 [n_cap][2]  x0 | y0 << 16, x1 | y1 << 16 (end exclusive, visible only)
 */
int32_t cgs_frame_buffer(const cgs_frame* frame, int32_t which, void** d_ptr, int64_t* count);

/* Stages of the hot path, for cgs_timing_read. */
#define CGS_STAGE_SELECT 0       /* level selection and segment lists (Sec. 3.3.2) */
#define CGS_STAGE_PROJECT 1      /* projection, tile rect, visible compaction, duplication into
                                    (tile, Gaussian) entries, SH colour */
#define CGS_STAGE_DUPLICATE 2    /* tile ranges, scatter of the entries into them */
#define CGS_STAGE_SORT 3         /* per-tile depth sort */
#define CGS_STAGE_RENDER 4       /* front-to-back compositing (Eq. 1) */
#define CGS_STAGE_RENDER_BWD 5   /* compositing backward */
#define CGS_STAGE_PROJECT_BWD 6  /* projection and colour backward */
#define CGS_STAGE_LOSS 7         /* L1 loss */
#define CGS_N_STAGES 8

/* Benchmark instrumentation.  While enabled (on != 0), every stage launched by
 * cgs_render_forward, cgs_render_backward and cgs_l1_loss is bracketed by a pair of CUDA
 * events recorded on the caller's stream (library-owned events, created on first use, at
 * most 256 pairs per stage between reads).  cgs_timing_read synchronizes those events and
 * returns, per stage, the summed milliseconds and the number of bracketed launches since the
 * previous read.  Not for use during stream capture. */
int32_t cgs_timing_enable(int32_t on);
int32_t cgs_timing_read(double* ms /*[CGS_N_STAGES]*/, int64_t* count /*[CGS_N_STAGES]*/);

/* Measured issue-rate peaks of the current device, for roofline denominators (instrumentation;
 * the paper has no counterpart).  Runs three loops on every SM -- scalar FP32 fused
 * multiply-adds, packed FP32x2 fused multiply-adds, and base-2 exponentials (ex2.approx, the
 * compositing kernels' one transcendental per pair) -- each timed with CUDA events on
 * `stream` (best of three after a warm-up), and SYNCHRONISES the stream.  rates[0] = FP32 lane
 * operations per second (one FMA instruction of one lane = 1), rates[1] = the same counted
 * from the packed loop (one packed instruction of one lane = 2), rates[2] = exponentials per
 * second.  n_rates >= 3.  d_scratch is a device array of at least (SM count x 2048) floats
 * that the loops overwrite. */
int32_t cgs_measure_peaks(double* rates, int32_t n_rates, float* d_scratch, int64_t scratch_floats, void* stream);

/* Test hook: d_g[i] = 2^d_p[i] evaluated exactly as both compositing kernels evaluate the
 * Gaussian falloff of Eq. 1 (the hardware base-2 exponential, results below the smallest normal
 * FP32 value flushed to zero), so that tests can bound its error.  n >= 0 values; asynchronous. */
int32_t cgs_debug_exp2(const float* d_p, int64_t n, float* d_g, void* stream);

/* Number of CUDA kernels this library has launched in the process so far (host counter). */
int64_t cgs_kernel_launches(void);

/* cgs_render_forward that also counts, for every scene Gaussian, the pixels (over all views of
 * the frame) whose compositing blends it: d_hits[scene index] += that count.  d_hits is a
 * device array of scene->n uint32 owned by the caller and only added to (clear it to start a
 * count; accumulate over frames to count over many views).  The image, T and n_contrib
 * outputs are those of cgs_render_forward.  The counts are the hit term of the significance
 * ranking that builds the detail levels (Sec. 3.3.1, cgs_generate_levels). */
int32_t cgs_render_forward_hits(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                                const cgs_camera* d_cams, const int32_t* d_view_block, const int8_t* d_levels,
                                float* d_image, float* d_final_T, uint32_t* d_n_contrib, uint32_t* d_hits,
                                void* stream);

/* ---- Detail levels (Sec. 3.3.1) ---------------------------------------------------------
 * Input: a block-grouped scene of n rows, block b = rows [d_block_offset[b],
 * d_block_offset[b + 1]) (offsets non-decreasing, offset[0] = 0, offset[n_blocks] = n: what
 * cgs_partition writes).  Inside every block the rows are ranked by descending significance
 *     s = o * ((s_x * s_y) * s_z)                   (d_hits == NULL: opacity x volume)
 *     s = (float)h * (o * ((s_x * s_y) * s_z))      (d_hits: pixel hit counts per row, from
 *                                                    cgs_render_forward_hits)
 * in FP32, this order; NaN ranks as -inf, -0 as +0; equal scores by increasing row.  Level l
 * of a block of K rows keeps the first floor(K * rates[l]) rows (FP64 product, rates in
 * [0, 1]), so the levels are nested prefixes of one order (the paper prunes with a
 * compressor at several rates; level 0 is the finest here).
 * Outputs: d_perm[n], position offset[b] + r = row of rank r in block b (gather the
 * attributes with cgs_gather_rows), and d_level_count[n_blocks][n_levels]; the new scene's
 * level_offset[b][l] is offset[b] for every l.  d_scale is [n][4] FP32, or [n][4] FP16 with
 * attr_fp16 = 1.  n_blocks <= CGS_PARTITION_MAX_BLOCKS, n_levels <= CGS_MAX_LEVELS.
 * Asynchronous; cgs_levels_status reads the device status. */
#define CGS_MAX_LEVELS 16
int64_t cgs_levels_workspace_bytes(int64_t n, int32_t n_blocks);
int32_t cgs_generate_levels(const float* d_mean_opac, const void* d_scale, int32_t attr_fp16, int64_t n,
                            const int64_t* d_block_offset, int32_t n_blocks, const uint32_t* d_hits,
                            const double* rates, int32_t n_levels, int32_t* d_perm, int64_t* d_level_count,
                            void* d_ws, int64_t ws_bytes, void* stream);
/* Synchronises the stream; CGS_OK or CGS_ERR_SPIN_TIMEOUT for the last call on d_ws. */
int32_t cgs_levels_status(const void* d_ws, void* stream);

/* ---- SSIM of renders (Eq. 3, B1 pose assignment) ------------------------------------------
 * Mean SSIM of n_pairs image pairs ([channels][height][width] FP32 each, planar like the
 * render output): pair i compares a_i = d_a + i * a_stride (floats; a_stride = 0 compares
 * every b_i with the same a) and b_i = d_b + i * channels * height * width.  Per channel:
 * local means, variances and covariance under an 11 x 11 Gaussian window of sigma 1.5
 * (weights summing to 1, zero outside the image), the SSIM map
 * ((2 ma mb + C1)(2 sab + C2)) / ((ma^2 + mb^2 + C1)(sa^2 + sb^2 + C2)), C1 = 0.01^2,
 * C2 = 0.03^2, averaged over every pixel and channel -> d_ssim[i] (written).  d_map (may be
 * NULL) receives the per-pixel map averaged over channels, [n_pairs][height][width].  The
 * SSIM loss of Eq. 3 is 1 - d_ssim[i].  Asynchronous; n_pairs <= 65535. */
int32_t cgs_ssim(const float* d_a, int64_t a_stride, const float* d_b, int32_t n_pairs, int32_t channels,
                 int32_t width, int32_t height, float* d_ssim, float* d_map, void* stream);

/* ---- Pose-to-block assignment (Sec. 3.2.2, Eqs. 3-5) ----------------------------------------
 * For n_poses x n_blocks FP32 SSIM values d_ssim[i][j] (cgs_ssim of pose i's render with every
 * block against its render without block j) and the block of every pose's camera centre
 * d_pose_block[i] (cgs_pose_blocks; -1 for none): B1[i][j] = (1 - SSIM) > eps (Eq. 3, FP32),
 * B2[i][j] = (d_pose_block[i] == j) (Eq. 4), B = B1 or B2 (Eq. 5).  Each of d_b1, d_b2, d_b
 * (uint8 [n_poses][n_blocks], 0 or 1) may be NULL, not all three.  Asynchronous. */
int32_t cgs_pose_assign(const float* d_ssim, const int32_t* d_pose_block, int32_t n_poses, int32_t n_blocks,
                        float eps, uint8_t* d_b1, uint8_t* d_b2, uint8_t* d_b, void* stream);

/* ---- Block partition of a scene (Sec. 3.2.2, Eqs. 2 and 4) --------------------------------
 * Positions are rows of `stride` floats with x, y, z first (stride 4 reads the mean_opac rows
 * of a scene directly; stride 3 reads plain xyz).  pmin, pmax (3 floats each) and grid
 * (3 int32) are HOST pointers; every other pointer is device memory owned by the caller.
 *
 *   normalisation  h = 2 (p - pmin) / (pmax - pmin) - 1, per axis (the foreground box
 *                  [pmin, pmax] maps to [-1, 1]^3); pmax > pmin, finite, on every axis
 *   contraction    Eq. 2: h if ||h||_inf <= 1, else (2 - 1/||h||_inf) h / ||h||_inf, a point
 *                  of the open cube (-2, 2)^3
 *   grid           the contracted cube split evenly into grid[0] x grid[1] x grid[2] blocks
 *                  (1..CGS_PARTITION_MAX_CELLS cells per axis, at most
 *                  CGS_PARTITION_MAX_BLOCKS blocks): along an axis of g cells the inner bounds
 *                  are b_i = 4 i / g - 2 and a coordinate c is in cell i when b_i <= c < b_{i+1}
 *                  (the outer cells are open to -inf and +inf); block = ix + grid[0] (iy +
 *                  grid[1] iz); -1 when the contracted point is not finite
 * Every value that decides a block is FP32, one rounding per operation, in the order above.
 * Invalid arguments return CGS_ERR_INVALID_ARGUMENT before any device work. */
#define CGS_PARTITION_MAX_CELLS 64
#define CGS_PARTITION_MAX_BLOCKS 1024

/* Contracted positions d_out[n][3] (Eq. 2 after the normalisation).  Asynchronous. */
int32_t cgs_contract(const float* d_pos, int64_t n, int64_t stride, const float* pmin, const float* pmax,
                     float* d_out, void* stream);

/* Eq. 4 (B2): d_block[i] = block of camera centre i, the same mapping as a Gaussian's. */
int32_t cgs_pose_blocks(const float* d_pos, int64_t n, int64_t stride, const float* pmin, const float* pmax,
                        const int32_t* grid, int32_t* d_block, void* stream);

/* Bytes of device workspace cgs_partition needs for n points and this grid; -1 if invalid. */
int64_t cgs_partition_workspace_bytes(int64_t n, const int32_t* grid);

/* The partition of n < 2^31 Gaussians: d_block[n] (block per Gaussian, -1 for none),
 * d_block_offset[n_blocks + 1] (first grouped position of every block; the last entry is the
 * number of grouped Gaussians, n minus those with no block) and, if d_perm is not NULL,
 * d_perm[offset[n_blocks]]: the scene index of every grouped position, block 0's Gaussians
 * first, each block in increasing scene index (a stable grouping, Sec. 3.2.2's G_Kj), and,
 * if d_rank is not NULL, d_rank[n]: the grouped position of every scene index (-1 for none),
 * the inverse permutation.
 * d_ws holds at least cgs_partition_workspace_bytes(n, grid) bytes, 256-byte aligned, not
 * shared with a concurrent call.  Asynchronous; read the device status with
 * cgs_partition_status.  Returns CGS_ERR_WORKSPACE_TOO_SMALL for a short workspace. */
int32_t cgs_partition(const float* d_pos, int64_t n, int64_t stride, const float* pmin, const float* pmax,
                      const int32_t* grid, int32_t* d_block, int64_t* d_block_offset, int32_t* d_perm,
                      int32_t* d_rank, void* d_ws, int64_t ws_bytes, void* stream);

/* Synchronises the stream and returns CGS_OK or CGS_ERR_SPIN_TIMEOUT (a bounded wait of the
 * offsets scan gave up; outputs invalid) for the last cgs_partition on d_ws. */
int32_t cgs_partition_status(const void* d_ws, void* stream);

/* Row gather: dst row r = src row d_perm[r], for n_rows rows of row_bytes bytes (a multiple
 * of 4).  Moves any per-Gaussian attribute array (FP32 or FP16) into the grouped order, so
 * that each block's Gaussians form one contiguous segment.  src and dst must not overlap;
 * every d_perm value must be a valid row of src.  Asynchronous. */
int32_t cgs_gather_rows(const void* d_src, void* d_dst, int64_t row_bytes, const int32_t* d_perm, int64_t n_rows,
                        void* stream);

/* Row scatter, the inverse move: dst row d_rank[r] = src row r for n_rows rows (rows with a
 * negative rank are skipped).  With the d_rank of cgs_partition it produces the grouped order
 * while reading src sequentially (the faster of the two for rows of 16 bytes).  Every
 * non-negative rank must be a valid row of dst and distinct.  Asynchronous. */
int32_t cgs_scatter_rows(const void* d_src, void* d_dst, int64_t row_bytes, const int32_t* d_rank, int64_t n_rows,
                         void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CGS_H */
