// Host entry points of libcgs (include/cgs.h): argument checks, the frame workspace layout
// and the launch sequence of the hot path.  Every call only enqueues work on the caller's
// stream; nothing here allocates device memory.
#include <string.h>

#include "common.cuh"

namespace cgs {
void launch_select(const Layout& L, const cgs_scene& S, const cgs_camera* cams, const int32_t* view_block,
                   const int8_t* levels, const cgs_config& cfg, cudaStream_t st);
void launch_lod_levels(const cgs_scene& S, const cgs_config& cfg, const cgs_camera* cams, int n_views,
                       int8_t* levels, cudaStream_t st);
void launch_block_bounds(const cgs_scene& S, double n_mad, float* aabb, cudaStream_t st);
void launch_project(const Layout& L, const cgs_scene& S, const cgs_camera* cams, float near_z, int n_sm,
                    cudaStream_t st);
int launch_bin(const Layout& L, int n_sm, cudaStream_t st);
int launch_tile_sort(const Layout& L, int n_sm, cudaStream_t st);
bool launch_render_fwd(const Layout& L, const cgs_config& c, float* img, float* T, uint32_t* nc, cudaStream_t st);
bool launch_render_bwd(const Layout& L, const cgs_config& c, const float* dimg, const float* T, const uint32_t* nc,
                       const L1In* l1, cudaStream_t st);
void launch_project_bwd(const Layout& L, const cgs_scene& S, const cgs_camera* cams, float near_z, float* g_mo,
                        float* g_sc, float* g_q, float* g_sh, long long* g_index, int n_sm, cudaStream_t st);
void launch_l1(const float* img, const float* tgt, long long n, float* loss, float* grad, int n_sm, cudaStream_t st);
void launch_l1_u8(const float* img, const uint8_t* tgt, long long n, float* loss, float* grad, int n_sm,
                  cudaStream_t st);
void launch_debug_exp2(const float* p, long long n, float* g, int n_sm, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// launch counting and optional per-stage event timing
// ---------------------------------------------------------------------------------------
static long long g_launches = 0;
static void counted(int n) { __atomic_add_fetch(&g_launches, (long long)n, __ATOMIC_RELAXED); }

constexpr int TIMING_SLOTS = 256;
struct StageTiming {
    bool on = false;
    bool created = false;
    cudaEvent_t ev[CGS_N_STAGES][TIMING_SLOTS][2];
    int used[CGS_N_STAGES] = {0};
};
static StageTiming g_timing;

struct StageScope {
    int stage;
    cudaStream_t st;
    int slot;
    StageScope(int s, cudaStream_t stream) : stage(s), st(stream), slot(-1)
    {
        if (g_timing.on && g_timing.created && g_timing.used[s] < TIMING_SLOTS) {
            slot = g_timing.used[s]++;
            cudaEventRecord(g_timing.ev[s][slot][0], st);
        }
    }
    ~StageScope()
    {
        if (slot >= 0) cudaEventRecord(g_timing.ev[stage][slot][1], st);
    }
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
    char* base;
    size_t off;
    template <typename T>
    T* take(long long count)
    {
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off = align_up(off + (size_t)count * sizeof(T));
        return p;
    }
};

// Fills L from the frame dimensions; returns false if they are invalid.
static bool make_layout(const cgs_frame* f, Layout* L, size_t* bytes)
{
    if (!f || (f->flags & ~CGS_FRAME_NO_PAIR_COUNT) != 0 || f->n_views < 1 || f->n_views > 65535 || f->width < 1 ||
        f->height < 1 ||
        (f->tile != 16 && f->tile != 8) || f->n_blocks < 1 || f->n_cap < 1 || f->n_cap >= (1ll << 31) ||
        f->k_cap < 1 || f->k_cap >= (1ll << 30))
        return false;
    Layout l;
    memset(&l, 0, sizeof(l));
    l.V = f->n_views;
    l.W = f->width;
    l.H = f->height;
    l.B = f->tile;
    l.tiles_x = (f->width + f->tile - 1) / f->tile;
    l.tiles_y = (f->height + f->tile - 1) / f->tile;
    if (l.tiles_x > 65535 || l.tiles_y > 65535) return false;
    l.T = l.tiles_x * l.tiles_y;
    if ((unsigned long long)l.V * (unsigned long long)l.T >= (1ull << 32)) return false;
    l.NB = f->n_blocks;
    l.n_cap = f->n_cap;
    l.k_cap = f->k_cap;
    const long long vt = (long long)l.V * l.T;
    l.tsub_sh = vt <= TSUB_MAX_TILES ? 2 : 0;
    static_assert(TSUB == 4, "tsub_sh is log2 of TSUB");
    const long long vts = vt << l.tsub_sh;
    const long long scan_tiles_vt = (vts + SCAN_TILE - 1) / SCAN_TILE;

    Carver c{(char*)f->ws, 0};
    l.hdr = c.take<Header>(1);
    l.scan_lb = c.take<unsigned long long>(scan_tiles_vt);
    l.tcnt = c.take<uint32_t>(vts);
    l.tcur = c.take<uint32_t>(vts);
    l.sel_done = c.take<uint32_t>(l.V);
    l.zero_bytes = c.off;
    l.ranges = c.take<uint32_t>(2 * vt);
    l.ssub = c.take<uint32_t>(vts);
    l.view_base = c.take<uint32_t>(l.V + 1);
    l.view_cnt = c.take<uint32_t>(l.V);
    l.n_seg = c.take<uint32_t>(l.V);
    l.seg_base = c.take<uint32_t>((long long)l.V * (l.NB + 1));
    l.seg_off = c.take<long long>((long long)l.V * l.NB);
    l.seg_blk = c.take<int32_t>((long long)l.V * l.NB);
    l.levels = c.take<int8_t>((long long)l.V * l.NB);
    l.rec = c.take<float4>(3 * l.n_cap);
    l.rect = c.take<uint2>(l.n_cap);
    l.tt = c.take<uint32_t>(l.n_cap);
    l.gidx = c.take<uint32_t>(l.n_cap);
    l.pkey = c.take<unsigned long long>(l.n_cap);
    l.vis = c.take<uint32_t>(l.n_cap);
    l.eraw = c.take<unsigned long long>(l.k_cap);
    l.ekey = c.take<unsigned long long>(l.k_cap);
    l.tval = c.take<uint32_t>(l.k_cap);
    l.tkey = c.take<uint32_t>(l.k_cap);
    l.big = c.take<uint32_t>(vt);
    l.gs = c.take<float4>(3 * l.n_cap);
    // per tile t and warp w: NW words per 32 entries of the tile plus one, at NW * (start_t / 32 + t)
    const int nw = (l.B * l.B) / 64;
    l.cbits_words = (long long)nw * (l.k_cap / 32 + vt + 1);
    l.cbits = c.take<uint32_t>(l.cbits_words);
    l.hits = nullptr;
    l.count_pairs = (f->flags & CGS_FRAME_NO_PAIR_COUNT) ? 0 : 1;
    *L = l;
    *bytes = c.off;
    return true;
}

static int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cache[dev] = n;
    }
    return cache[dev];
}

static bool scene_ok(const cgs_scene* s)
{
    return s && s->n >= 0 && s->n < (1ll << 31) && s->sh_degree >= 0 && s->sh_degree <= 3 && s->n_blocks >= 1 &&
           s->n_blocks < (1 << 20) &&
           (s->attr_fp16 == 0 || s->attr_fp16 == 1) &&
           s->n_levels >= 1 && s->mean_opac && s->scale && s->quat && s->sh && s->level_offset && s->level_count;
}

static bool config_ok(const cgs_config* c, int tile)
{
    if (!c || c->tile != tile) return false;
    if (!(c->near_z > 0.0f)) return false;
    const int b = c->batch;
    if (b != 32 && b != 64 && b != 128 && b != 256) return false;
    return b <= tile * tile;
}

// shared with the entry points of the other files (partition.cu)
void count_launches(int n) { counted(n); }
int device_sm_count() { return sm_count(); }

}  // namespace cgs

using namespace cgs;

extern "C" {

int32_t cgs_version(void) { return 1; }

const char* cgs_status_string(int32_t code)
{
    switch (code) {
        case CGS_OK: return "ok";
        case CGS_ERR_INVALID_ARGUMENT: return "invalid argument";
        case CGS_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
        case CGS_ERR_CAPACITY: return "capacity exceeded (selected Gaussians or tile entries)";
        case CGS_ERR_SPIN_TIMEOUT: return "a bounded inter-block wait gave up";
        case CGS_ERR_CUDA: return "CUDA error";
        case CGS_ERR_UNSUPPORTED: return "unsupported configuration";
        case CGS_ERR_TOO_LARGE: return "request exceeds the limits of the static-workspace entry point";
    }
    return "unknown status";
}

int64_t cgs_frame_workspace_bytes(int32_t n_views, int32_t width, int32_t height, int32_t tile, int32_t n_blocks,
                                  int64_t n_cap, int64_t k_cap)
{
    cgs_frame f;
    memset(&f, 0, sizeof(f));
    f.n_views = n_views;
    f.width = width;
    f.height = height;
    f.tile = tile;
    f.n_blocks = n_blocks;
    f.n_cap = n_cap;
    f.k_cap = k_cap;
    Layout L;
    size_t bytes = 0;
    if (!make_layout(&f, &L, &bytes)) return 0;
    return (int64_t)bytes;
}

int64_t cgs_block_bounds_workspace_bytes(int64_t n)
{
    (void)n;
    return 0;
}

int32_t cgs_block_bounds(const cgs_scene* scene, double n_mad, float* d_aabb, void* d_ws, int64_t ws_bytes,
                         void* stream)
{
    (void)d_ws;
    (void)ws_bytes;
    if (!scene_ok(scene) || !d_aabb || !(n_mad >= 0.0)) return CGS_ERR_INVALID_ARGUMENT;
    launch_block_bounds(*scene, n_mad, d_aabb, (cudaStream_t)stream);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

int32_t cgs_lod_select(const cgs_scene* scene, const cgs_config* cfg, const cgs_camera* d_cams, int32_t n_views,
                       int8_t* d_levels, void* stream)
{
    if (!scene_ok(scene) || !scene->block_aabb || !scene->block_cell || !cfg || !d_cams || !d_levels ||
        n_views < 1 || !(cfg->near_z > 0.0f))
        return CGS_ERR_INVALID_ARGUMENT;
    launch_lod_levels(*scene, *cfg, d_cams, n_views, d_levels, (cudaStream_t)stream);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

static int32_t render_forward(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                              const cgs_camera* d_cams, const int32_t* d_view_block, const int8_t* d_levels,
                              float* d_image, float* d_final_T, uint32_t* d_n_contrib, uint32_t* d_hits, void* stream)
{
    Layout L;
    size_t bytes = 0;
    if (!make_layout(frame, &L, &bytes) || !frame->ws) return CGS_ERR_INVALID_ARGUMENT;
    L.hits = d_hits;
    if ((size_t)frame->ws_bytes < bytes) return CGS_ERR_WORKSPACE_TOO_SMALL;
    if (!scene_ok(scene) || scene->n_blocks != frame->n_blocks || !config_ok(cfg, frame->tile) || !d_cams ||
        !d_image || !d_final_T || !d_n_contrib)
        return CGS_ERR_INVALID_ARGUMENT;
    if (!d_levels && !d_view_block && (!scene->block_aabb || !scene->block_cell)) return CGS_ERR_INVALID_ARGUMENT;
    if (cfg->lod_mode != CGS_LOD_BLOCK && cfg->lod_mode != CGS_LOD_POINT) return CGS_ERR_INVALID_ARGUMENT;
    // the point-wise test applies only when the renderer chooses levels itself
    L.lod_mode = (d_levels || d_view_block) ? CGS_LOD_BLOCK : cfg->lod_mode;
    L.lod_d1 = (float)cfg->lod_dist[0];
    L.lod_d2 = (float)cfg->lod_dist[1];
    cudaStream_t st = (cudaStream_t)stream;
    const int n_sm = sm_count();
    if (cudaMemsetAsync(frame->ws, 0, L.zero_bytes, st) != cudaSuccess) return CGS_ERR_CUDA;
    {
        StageScope s(CGS_STAGE_SELECT, st);
        launch_select(L, *scene, d_cams, d_view_block, d_levels, *cfg, st);
        counted(1);
    }
    {
        StageScope s(CGS_STAGE_PROJECT, st);
        launch_project(L, *scene, d_cams, cfg->near_z, n_sm, st);
        counted(1);
    }
    {
        StageScope s(CGS_STAGE_DUPLICATE, st);
        counted(launch_bin(L, n_sm, st));
    }
    {
        StageScope s(CGS_STAGE_SORT, st);
        const int n = launch_tile_sort(L, n_sm, st);
        if (n < 0) return CGS_ERR_CUDA;
        counted(n);
    }
    {
        StageScope s(CGS_STAGE_RENDER, st);
        if (!launch_render_fwd(L, *cfg, d_image, d_final_T, d_n_contrib, st)) return CGS_ERR_UNSUPPORTED;
        counted(1);
    }
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

int32_t cgs_render_forward(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                           const cgs_camera* d_cams, const int32_t* d_view_block, const int8_t* d_levels,
                           float* d_image, float* d_final_T, uint32_t* d_n_contrib, void* stream)
{
    return render_forward(scene, frame, cfg, d_cams, d_view_block, d_levels, d_image, d_final_T, d_n_contrib,
                          nullptr, stream);
}

int32_t cgs_render_forward_hits(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                                const cgs_camera* d_cams, const int32_t* d_view_block, const int8_t* d_levels,
                                float* d_image, float* d_final_T, uint32_t* d_n_contrib, uint32_t* d_hits,
                                void* stream)
{
    if (!d_hits) return CGS_ERR_INVALID_ARGUMENT;
    return render_forward(scene, frame, cfg, d_cams, d_view_block, d_levels, d_image, d_final_T, d_n_contrib,
                          d_hits, stream);
}

// l1 == NULL: dL/dimage from d_dL_dimage; else the fused L1 loss (d_dL_dimage unused).
static int32_t render_backward(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                               const cgs_camera* d_cams, const float* d_dL_dimage, const float* d_final_T,
                               const uint32_t* d_n_contrib, float* d_g_mean_opac, float* d_g_scale, float* d_g_quat,
                               float* d_g_sh, int64_t* d_g_index, const L1In* l1, void* stream)
{
    Layout L;
    size_t bytes = 0;
    if (!make_layout(frame, &L, &bytes) || !frame->ws) return CGS_ERR_INVALID_ARGUMENT;
    if ((size_t)frame->ws_bytes < bytes) return CGS_ERR_WORKSPACE_TOO_SMALL;
    if (!scene_ok(scene) || scene->n_blocks != frame->n_blocks || !config_ok(cfg, frame->tile) || !d_cams ||
        (!l1 && !d_dL_dimage) || !d_final_T || !d_n_contrib || !d_g_mean_opac || !d_g_scale || !d_g_quat ||
        !d_g_sh)
        return CGS_ERR_INVALID_ARGUMENT;
    if (l1 && cfg->exact) return CGS_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const int n_sm = sm_count();
    {
        StageScope s(CGS_STAGE_RENDER_BWD, st);
        if (!launch_render_bwd(L, *cfg, d_dL_dimage, d_final_T, d_n_contrib, l1, st)) return CGS_ERR_UNSUPPORTED;
        counted(1);
    }
    {
        StageScope s(CGS_STAGE_PROJECT_BWD, st);
        launch_project_bwd(L, *scene, d_cams, cfg->near_z, d_g_mean_opac, d_g_scale, d_g_quat, d_g_sh,
                           reinterpret_cast<long long*>(d_g_index), n_sm, st);
        counted(1);
    }
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

int32_t cgs_render_backward(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                            const cgs_camera* d_cams, const float* d_dL_dimage, const float* d_final_T,
                            const uint32_t* d_n_contrib, float* d_g_mean_opac, float* d_g_scale, float* d_g_quat,
                            float* d_g_sh, void* stream)
{
    return render_backward(scene, frame, cfg, d_cams, d_dL_dimage, d_final_T, d_n_contrib, d_g_mean_opac, d_g_scale,
                           d_g_quat, d_g_sh, nullptr, nullptr, stream);
}

int32_t cgs_render_backward_packed(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                                   const cgs_camera* d_cams, const float* d_dL_dimage, const float* d_final_T,
                                   const uint32_t* d_n_contrib, float* d_g_mean_opac, float* d_g_scale,
                                   float* d_g_quat, float* d_g_sh, int64_t* d_g_index, void* stream)
{
    if (!d_g_index) return CGS_ERR_INVALID_ARGUMENT;
    return render_backward(scene, frame, cfg, d_cams, d_dL_dimage, d_final_T, d_n_contrib, d_g_mean_opac, d_g_scale,
                           d_g_quat, d_g_sh, d_g_index, nullptr, stream);
}

int32_t cgs_render_backward_l1(const cgs_scene* scene, const cgs_frame* frame, const cgs_config* cfg,
                               const cgs_camera* d_cams, const float* d_image, const void* d_target,
                               int32_t target_u8, const float* d_final_T, const uint32_t* d_n_contrib,
                               float* d_loss, float* d_g_mean_opac, float* d_g_scale, float* d_g_quat,
                               float* d_g_sh, int64_t* d_g_index, void* stream)
{
    if (!frame || !d_image || !d_target || !d_loss || (target_u8 != 0 && target_u8 != 1) || frame->n_views < 1 ||
        frame->width < 1 || frame->height < 1)
        return CGS_ERR_INVALID_ARGUMENT;
    const long long count = 3LL * frame->n_views * frame->width * frame->height;
    L1In l1;
    l1.img = d_image;
    l1.tgt = d_target;
    l1.loss = d_loss;
    l1.inv = 1.0f / (float)count;  // the FP32 quotient cgs_l1_loss forms on the device
    l1.u8 = target_u8;
    return render_backward(scene, frame, cfg, d_cams, nullptr, d_final_T, d_n_contrib, d_g_mean_opac, d_g_scale,
                           d_g_quat, d_g_sh, d_g_index, &l1, stream);
}

int32_t cgs_l1_loss(const float* d_img, const float* d_target, int64_t count, float* d_loss, float* d_grad,
                    void* stream)
{
    if (!d_img || !d_target || !d_loss || !d_grad || count < 1) return CGS_ERR_INVALID_ARGUMENT;
    {
        StageScope s(CGS_STAGE_LOSS, (cudaStream_t)stream);
        launch_l1(d_img, d_target, count, d_loss, d_grad, sm_count(), (cudaStream_t)stream);
        counted(1);
    }
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

int32_t cgs_l1_loss_u8(const float* d_img, const uint8_t* d_target, int64_t count, float* d_loss, float* d_grad,
                       void* stream)
{
    if (!d_img || !d_target || !d_loss || !d_grad || count < 1) return CGS_ERR_INVALID_ARGUMENT;
    {
        StageScope s(CGS_STAGE_LOSS, (cudaStream_t)stream);
        launch_l1_u8(d_img, d_target, count, d_loss, d_grad, sm_count(), (cudaStream_t)stream);
        counted(1);
    }
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

int32_t cgs_frame_status(const cgs_frame* frame, int32_t* status, int64_t* counts, void* stream)
{
    Layout L;
    size_t bytes = 0;
    if (!make_layout(frame, &L, &bytes) || !frame->ws) return CGS_ERR_INVALID_ARGUMENT;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CGS_ERR_CUDA;
    Header h;
    if (cudaMemcpy(&h, L.hdr, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return CGS_ERR_CUDA;
    int32_t code = CGS_OK;
    if (h.status & ST_SPIN) code = CGS_ERR_SPIN_TIMEOUT;
    else if (h.status & ST_CAPACITY) code = CGS_ERR_CAPACITY;
    else if (h.status & ST_UNSUPPORTED) code = CGS_ERR_UNSUPPORTED;
    if (status) *status = code;
    if (counts) {
        counts[0] = (int64_t)h.n_sel_raw;
        counts[1] = (int64_t)h.n_vis;
        counts[2] = (int64_t)h.k_total;
        counts[3] = (int64_t)h.pairs_fwd;
        counts[4] = (int64_t)h.pairs_bwd;
        counts[5] = (int64_t)h.spin_giveups;
        counts[6] = (int64_t)h.steps_fwd;
        counts[7] = (int64_t)h.steps_useful;
    }
    return code;
}

int32_t cgs_timing_enable(int32_t on)
{
    if (on && !g_timing.created) {
        for (int s = 0; s < CGS_N_STAGES; s++)
            for (int k = 0; k < TIMING_SLOTS; k++)
                for (int e = 0; e < 2; e++)
                    if (cudaEventCreate(&g_timing.ev[s][k][e]) != cudaSuccess) return CGS_ERR_CUDA;
        g_timing.created = true;
    }
    g_timing.on = on != 0;
    for (int s = 0; s < CGS_N_STAGES; s++) g_timing.used[s] = 0;
    return CGS_OK;
}

int32_t cgs_timing_read(double* ms, int64_t* count)
{
    for (int s = 0; s < CGS_N_STAGES; s++) {
        double acc = 0.0;
        for (int k = 0; k < g_timing.used[s]; k++) {
            if (cudaEventSynchronize(g_timing.ev[s][k][1]) != cudaSuccess) return CGS_ERR_CUDA;
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, g_timing.ev[s][k][0], g_timing.ev[s][k][1]) != cudaSuccess) return CGS_ERR_CUDA;
            acc += t;
        }
        if (ms) ms[s] = acc;
        if (count) count[s] = g_timing.used[s];
        g_timing.used[s] = 0;
    }
    return CGS_OK;
}

int64_t cgs_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int32_t cgs_debug_exp2(const float* d_p, int64_t n, float* d_g, void* stream)
{
    if (!d_p || !d_g || n < 0) return CGS_ERR_INVALID_ARGUMENT;
    if (n == 0) return CGS_OK;
    launch_debug_exp2(d_p, n, d_g, sm_count(), (cudaStream_t)stream);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

int32_t cgs_frame_buffer(const cgs_frame* frame, int32_t which, void** d_ptr, int64_t* count)
{
    Layout L;
    size_t bytes = 0;
    if (!make_layout(frame, &L, &bytes) || !frame->ws || !d_ptr) return CGS_ERR_INVALID_ARGUMENT;
    void* p = nullptr;
    int64_t n = 0;
    switch (which) {
        case 0: p = L.tkey; n = L.k_cap; break;
        case 1: p = L.tval; n = L.k_cap; break;
        case 2: p = L.ranges; n = (int64_t)L.V * L.T; break;
        case 3: p = L.gidx; n = L.n_cap; break;
        case 4: p = L.rec; n = L.n_cap; break;
        case 5: p = L.tt; n = L.n_cap; break;
        case 6: p = L.view_base; n = L.V + 1; break;
        case 7: p = L.vis; n = L.n_cap; break;
        case 8: p = L.pkey; n = L.n_cap; break;
        case 9: p = L.rect; n = L.n_cap; break;
        default: return CGS_ERR_INVALID_ARGUMENT;
    }
    *d_ptr = p;
    if (count) *count = n;
    return CGS_OK;
}

}  // extern "C"
