// Entry points around the hot path: uploading a block-partitioned scene into caller-owned
// device memory (Sec. 3.1's Gaussian attributes with Sec. 3.3.2's per-block detail levels),
// the pose-to-block decision of Eqs. 3-5 (Sec. 3.2.2), and the autotuner that times the real
// rendering step for each tile size and compositing batch depth.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace cgs {

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SceneCarve {
    size_t mo, sc, q, sh, lo, lc, cell, aabb, total;
};

static bool scene_carve(int64_t n, int32_t deg, int32_t nb, int32_t nl, int32_t fp16, SceneCarve* c)
{
    if (n < 0 || n >= (1ll << 31) || deg < 0 || deg > 3 || nb < 1 || nb >= (1 << 20) || nl < 1 ||
        nl > CGS_MAX_LEVELS || (fp16 != 0 && fp16 != 1))
        return false;
    const size_t e = fp16 ? 2 : 4, nco = (size_t)(deg + 1) * (deg + 1);
    size_t off = 0;
    c->mo = off; off = up256(off + (size_t)n * 16);
    c->sc = off; off = up256(off + (size_t)n * 4 * e);
    c->q = off; off = up256(off + (size_t)n * 4 * e);
    c->sh = off; off = up256(off + (size_t)n * nco * 3 * e);
    c->lo = off; off = up256(off + (size_t)nb * nl * 8);
    c->lc = off; off = up256(off + (size_t)nb * nl * 8);
    c->cell = off; off = up256(off + (size_t)nb * 16);
    c->aabb = off; off = up256(off + (size_t)nb * 24);
    c->total = off;
    return true;
}

// Eqs. 3-5 for a [n_poses][n_blocks] grid.
__global__ void __launch_bounds__(256) k_pose_assign(const float* __restrict__ ssim, const int32_t* __restrict__ pose_block,
                                                     long long total, int nb, float eps, uint8_t* b1, uint8_t* b2,
                                                     uint8_t* b)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long i = t / nb;
        const int j = (int)(t - i * nb);
        const uint8_t x1 = (1.0f - ssim[t]) > eps ? 1 : 0;  // the SSIM loss of Eq. 3 against its threshold
        const uint8_t x2 = pose_block[i] == j ? 1 : 0;      // Eq. 4: the camera centre lies in block j
        if (b1) b1[t] = x1;
        if (b2) b2[t] = x2;
        if (b) b[t] = x1 | x2;                              // Eq. 5, read as a logical or
    }
}

__global__ void __launch_bounds__(256) k_fill(float* __restrict__ p, long long n, float v)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// The autotuner's candidates, in the order of the ms_out entries.
static const int32_t TUNE[CGS_TUNE_CANDIDATES][2] = {{16, 256}, {16, 128}, {16, 64}, {16, 32}, {8, 64}, {8, 32}};

struct TuneCarve {
    size_t frame, img, T, nc, dl, rows_mo, rows_sc, rows_q, rows_sh, rows_i, total;
    int64_t frame_bytes;
};

static bool tune_carve(int32_t V, int32_t W, int32_t H, int32_t nb, int64_t n_cap, int64_t k_cap, int32_t deg,
                       int32_t mode, TuneCarve* c)
{
    int64_t fb = 0;
    for (int k = 0; k < CGS_TUNE_CANDIDATES; k++) {
        const int64_t b = cgs_frame_workspace_bytes(V, W, H, TUNE[k][0], nb, n_cap, k_cap);
        if (b <= 0) return false;
        fb = std::max(fb, b);
    }
    if (deg < 0 || deg > 3 || (mode != CGS_TUNE_FORWARD && mode != CGS_TUNE_FORWARD_BACKWARD)) return false;
    const size_t px = (size_t)V * W * H, nco = (size_t)(deg + 1) * (deg + 1);
    size_t off = 0;
    c->frame = off; off = up256(off + (size_t)fb);
    c->img = off; off = up256(off + px * 3 * 4);
    c->T = off; off = up256(off + px * 4);
    c->nc = off; off = up256(off + px * 4);
    if (mode == CGS_TUNE_FORWARD_BACKWARD) {
        c->dl = off; off = up256(off + px * 3 * 4);
        c->rows_mo = off; off = up256(off + (size_t)n_cap * 16);
        c->rows_sc = off; off = up256(off + (size_t)n_cap * 16);
        c->rows_q = off; off = up256(off + (size_t)n_cap * 16);
        c->rows_sh = off; off = up256(off + (size_t)n_cap * nco * 12);
        c->rows_i = off; off = up256(off + (size_t)n_cap * 8);
    }
    c->total = off;
    c->frame_bytes = fb;
    return true;
}

// Cache lines "key tile batch" (key: device name and the caller's workload key, spaces
// replaced).  Returns true and the choice when the key is found.
static void cache_key_of(const char* user_key, char* out, size_t cap)
{
    int dev = 0;
    cudaDeviceProp p;
    const char* name = "unknown-device";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess) name = p.name;
    snprintf(out, cap, "%s|%s", name, user_key ? user_key : "");
    for (char* s = out; *s; s++)
        if (*s == ' ' || *s == '\t' || *s == '\n') *s = '_';
}

static bool cache_lookup(const char* path, const char* key, int32_t* tile, int32_t* batch)
{
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[600], k[520];
    int t = 0, b = 0;
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        if (sscanf(line, "%519s %d %d", k, &t, &b) == 3 && strcmp(k, key) == 0) {
            for (int c = 0; c < CGS_TUNE_CANDIDATES; c++)
                if (TUNE[c][0] == t && TUNE[c][1] == b) {
                    *tile = t;
                    *batch = b;
                    found = true;
                }
        }
    }
    fclose(f);
    return found;
}

}  // namespace cgs

using namespace cgs;

extern "C" int64_t cgs_scene_bytes(int64_t n, int32_t sh_degree, int32_t n_blocks, int32_t n_levels, int32_t attr_fp16)
{
    SceneCarve c;
    return scene_carve(n, sh_degree, n_blocks, n_levels, attr_fp16, &c) ? (int64_t)c.total : -1;
}

extern "C" int32_t cgs_scene_upload(cgs_scene* out, void* d_mem, int64_t mem_bytes, const float* h_mean_opac,
                                    const void* h_scale, const void* h_quat, const void* h_sh, int64_t n,
                                    int32_t sh_degree, int32_t attr_fp16, int32_t n_blocks, int32_t n_levels,
                                    const int64_t* h_level_offset, const int64_t* h_level_count,
                                    const float* h_block_cell, double n_mad, void* stream)
{
    SceneCarve c;
    if (!out || !d_mem || !scene_carve(n, sh_degree, n_blocks, n_levels, attr_fp16, &c) || !h_level_offset ||
        !h_level_count || !h_block_cell || (n > 0 && (!h_mean_opac || !h_scale || !h_quat || !h_sh)))
        return CGS_ERR_INVALID_ARGUMENT;
    if (mem_bytes < (int64_t)c.total) return CGS_ERR_WORKSPACE_TOO_SMALL;
    // the block table: every segment inside [0, n), and the blocks' segments ascending and apart
    int64_t prev_end = 0;
    for (int32_t b = 0; b < n_blocks; b++) {
        int64_t lo = INT64_MAX, hi = 0;
        for (int32_t l = 0; l < n_levels; l++) {
            const int64_t o = h_level_offset[(int64_t)b * n_levels + l], k = h_level_count[(int64_t)b * n_levels + l];
            if (o < 0 || k < 0 || o > n || k > n - o) return CGS_ERR_INVALID_ARGUMENT;
            if (k > 0) {
                lo = std::min(lo, o);
                hi = std::max(hi, o + k);
            }
        }
        if (hi > 0) {
            if (lo < prev_end) return CGS_ERR_INVALID_ARGUMENT;
            prev_end = hi;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)d_mem;
    const size_t e = attr_fp16 ? 2 : 4, nco = (size_t)(sh_degree + 1) * (sh_degree + 1);
    struct {
        size_t off;
        const void* src;
        size_t bytes;
    } copies[] = {{c.mo, h_mean_opac, (size_t)n * 16}, {c.sc, h_scale, (size_t)n * 4 * e},
                  {c.q, h_quat, (size_t)n * 4 * e}, {c.sh, h_sh, (size_t)n * nco * 3 * e},
                  {c.lo, h_level_offset, (size_t)n_blocks * n_levels * 8},
                  {c.lc, h_level_count, (size_t)n_blocks * n_levels * 8}, {c.cell, h_block_cell, (size_t)n_blocks * 16}};
    for (auto& cp : copies)
        if (cp.bytes && cudaMemcpyAsync(base + cp.off, cp.src, cp.bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return CGS_ERR_CUDA;
    cgs_scene s;
    memset(&s, 0, sizeof(s));
    s.mean_opac = (const float*)(base + c.mo);
    s.scale = (const float*)(base + c.sc);
    s.quat = (const float*)(base + c.q);
    s.sh = (const float*)(base + c.sh);
    s.n = n;
    s.sh_degree = sh_degree;
    s.n_blocks = n_blocks;
    s.n_levels = n_levels;
    s.attr_fp16 = attr_fp16;
    s.level_offset = (const int64_t*)(base + c.lo);
    s.level_count = (const int64_t*)(base + c.lc);
    s.block_cell = (const float*)(base + c.cell);
    s.block_aabb = (const float*)(base + c.aabb);
    if (n_mad >= 0.0) {
        const int32_t rc = cgs_block_bounds(&s, n_mad, (float*)(base + c.aabb), nullptr, 0, stream);
        if (rc != CGS_OK) return rc;
    } else if (cudaMemsetAsync(base + c.aabb, 0, (size_t)n_blocks * 24, st) != cudaSuccess) {
        return CGS_ERR_CUDA;
    }
    *out = s;
    return CGS_OK;
}

extern "C" int32_t cgs_pose_assign(const float* d_ssim, const int32_t* d_pose_block, int32_t n_poses, int32_t n_blocks,
                                   float eps, uint8_t* d_b1, uint8_t* d_b2, uint8_t* d_b, void* stream)
{
    if (n_poses < 0 || n_blocks < 1 || !(eps == eps) || (n_poses > 0 && (!d_ssim || !d_pose_block)) ||
        (!d_b1 && !d_b2 && !d_b))
        return CGS_ERR_INVALID_ARGUMENT;
    const long long total = (long long)n_poses * n_blocks;
    if (total == 0) return CGS_OK;
    const long long g = std::min<long long>((total + 255) / 256, (long long)device_sm_count() * 8);
    k_pose_assign<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(d_ssim, d_pose_block, total, n_blocks, eps, d_b1, d_b2,
                                                                 d_b);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

extern "C" int64_t cgs_autotune_workspace_bytes(int32_t n_views, int32_t width, int32_t height, int32_t n_blocks,
                                                int64_t n_cap, int64_t k_cap, int32_t sh_degree, int32_t mode)
{
    TuneCarve c;
    return tune_carve(n_views, width, height, n_blocks, n_cap, k_cap, sh_degree, mode, &c) ? (int64_t)c.total : -1;
}

extern "C" int32_t cgs_autotune(const cgs_scene* scene, const cgs_camera* d_cams, int32_t n_views, int32_t width,
                                int32_t height, const int32_t* d_view_block, const int8_t* d_levels, int64_t n_cap,
                                int64_t k_cap, int32_t mode, int32_t reps, void* d_ws, int64_t ws_bytes,
                                cgs_config* inout, float* ms_out, const char* cache_path, const char* cache_key,
                                void* stream)
{
    TuneCarve c;
    if (!scene || !d_cams || !inout || !d_ws || reps < 1 || reps > 1000 ||
        !tune_carve(n_views, width, height, scene->n_blocks, n_cap, k_cap, scene->sh_degree, mode, &c))
        return CGS_ERR_INVALID_ARGUMENT;
    if (ws_bytes < (int64_t)c.total) return CGS_ERR_WORKSPACE_TOO_SMALL;
    char key[520];
    cache_key_of(cache_key, key, sizeof(key));
    if (ms_out)
        for (int k = 0; k < CGS_TUNE_CANDIDATES; k++) ms_out[k] = -1.0f;
    if (cache_path && cache_lookup(cache_path, key, &inout->tile, &inout->batch)) return CGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)d_ws;
    float* img = (float*)(base + c.img);
    float* T = (float*)(base + c.T);
    uint32_t* nc = (uint32_t*)(base + c.nc);
    const long long px = (long long)n_views * width * height;
    if (mode == CGS_TUNE_FORWARD_BACKWARD) {
        // an upstream gradient of the size an L1 loss gives, on every pixel
        const long long g = std::min<long long>((3 * px + 255) / 256, (long long)device_sm_count() * 8);
        k_fill<<<(unsigned)g, 256, 0, st>>>((float*)(base + c.dl), 3 * px, 1.0f / (float)(3 * px));
        count_launches(1);
    }
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return CGS_ERR_CUDA;
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return CGS_ERR_CUDA;
    }
    int32_t rc = CGS_OK;
    int best = -1;
    float best_ms = 0.0f;
    int zeroed_tile = 0;
    for (int k = 0; k < CGS_TUNE_CANDIDATES && rc == CGS_OK; k++) {
        cgs_config cfg = *inout;
        cfg.tile = TUNE[k][0];
        cfg.batch = TUNE[k][1];
        cgs_frame f;
        memset(&f, 0, sizeof(f));
        f.ws = base + c.frame;
        f.ws_bytes = c.frame_bytes;
        f.n_views = n_views;
        f.width = width;
        f.height = height;
        f.tile = cfg.tile;
        f.n_blocks = scene->n_blocks;
        f.n_cap = n_cap;
        f.k_cap = k_cap;
        if (zeroed_tile != cfg.tile) {  // a frame workspace starts zero-filled (cgs_frame)
            if (cudaMemsetAsync(f.ws, 0, (size_t)c.frame_bytes, st) != cudaSuccess) { rc = CGS_ERR_CUDA; break; }
            zeroed_tile = cfg.tile;
        }
        auto step = [&]() -> int32_t {
            int32_t r = cgs_render_forward(scene, &f, &cfg, d_cams, d_view_block, d_levels, img, T, nc, stream);
            if (r == CGS_OK && mode == CGS_TUNE_FORWARD_BACKWARD)
                r = cgs_render_backward_packed(scene, &f, &cfg, d_cams, (const float*)(base + c.dl), T, nc,
                                               (float*)(base + c.rows_mo), (float*)(base + c.rows_sc),
                                               (float*)(base + c.rows_q), (float*)(base + c.rows_sh),
                                               (int64_t*)(base + c.rows_i), stream);
            return r;
        };
        int32_t r = step();  // warm-up; a candidate the frame cannot hold is not eligible
        if (r == CGS_ERR_UNSUPPORTED || r == CGS_ERR_INVALID_ARGUMENT) continue;
        if (r != CGS_OK) { rc = r; break; }
        int32_t status = CGS_OK;
        if (cgs_frame_status(&f, &status, nullptr, stream) == CGS_ERR_CUDA) { rc = CGS_ERR_CUDA; break; }
        if (status != CGS_OK) continue;
        std::vector<float> ms;
        for (int i = 0; i < reps && rc == CGS_OK; i++) {
            cudaEventRecord(ev[0], st);
            if ((r = step()) != CGS_OK) { rc = r; break; }
            cudaEventRecord(ev[1], st);
            if (cudaEventSynchronize(ev[1]) != cudaSuccess) { rc = CGS_ERR_CUDA; break; }
            float t = 0.0f;
            cudaEventElapsedTime(&t, ev[0], ev[1]);
            ms.push_back(t);
        }
        if (rc != CGS_OK) break;
        std::sort(ms.begin(), ms.end());
        const float med = ms[ms.size() / 2];
        if (ms_out) ms_out[k] = med;
        if (best < 0 || med < best_ms) {
            best = k;
            best_ms = med;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc != CGS_OK) return rc;
    if (best < 0) return CGS_ERR_CAPACITY;  // no candidate fit the frame capacities
    inout->tile = TUNE[best][0];
    inout->batch = TUNE[best][1];
    if (cache_path) {
        FILE* fo = fopen(cache_path, "a");
        if (fo) {
            fprintf(fo, "%s %d %d\n", key, inout->tile, inout->batch);
            fclose(fo);
        }
    }
    return CGS_OK;
}
