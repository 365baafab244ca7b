// Block-wise level-of-detail selection (stage a of the hot path, Sec. 3.3.2) and the MAD
// block bounds of Eq. 7.  FP64 throughout; compiled with -fmad=false so every expression is
// evaluated in the order written.
#include "common.cuh"

namespace cgs {

// Level of block b seen from camera c: -1 culled or empty, else 0..n_levels-1.
// Called by an aligned group of 8 lanes, lane `k` of the group handling box corner k; every
// lane of the warp must call it (inactive groups pass b < 0).  The corners of the box in
// front of the camera are projected; the block is visible if their screen bounding box
// overlaps the image; the block whose ground cell holds the camera centre is always kept;
// the level follows the minimum corner-to-camera distance.  sqrt is monotone and correctly
// rounded, so the minimum distance is sqrt of the minimum squared distance, bit for bit.
__device__ int lod_level8(const cgs_scene& S, int b, const cgs_camera& c, double near_z, double d1, double d2)
{
    const int k = threadIdx.x & 7;
    const bool active = b >= 0 && b < S.n_blocks && S.level_count[(long long)(b < 0 ? 0 : b) * S.n_levels] > 0;
    double e2 = INFINITY, xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    int front = 0;
    const double cp0 = (double)c.campos[0], cp1 = (double)c.campos[1], cp2 = (double)c.campos[2];
    if (active) {
        const float* bb = S.block_aabb + 6 * (long long)b;
        const double p0 = (double)bb[(k & 1) ? 3 : 0], p1 = (double)bb[(k & 2) ? 4 : 1], p2 = (double)bb[(k & 4) ? 5 : 2];
        const double e0 = p0 - cp0, ee1 = p1 - cp1, ee2 = p2 - cp2;
        e2 = (e0 * e0 + ee1 * ee1) + ee2 * ee2;
        double R[9], t[3];
        for (int i = 0; i < 9; i++) R[i] = (double)c.R[i];
        for (int i = 0; i < 3; i++) t[i] = (double)c.t[i];
        const double tx = ((R[0] * p0 + R[1] * p1) + R[2] * p2) + t[0];
        const double ty = ((R[3] * p0 + R[4] * p1) + R[5] * p2) + t[1];
        const double tz = ((R[6] * p0 + R[7] * p1) + R[8] * p2) + t[2];
        if (tz > near_z) {
            front = 1;
            const double u = ((double)c.fx * tx) / tz + (double)c.cx, v = ((double)c.fy * ty) / tz + (double)c.cy;
            xmin = xmax = u;
            ymin = ymax = v;
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        e2 = fmin(e2, __shfl_xor_sync(0xffffffffu, e2, o, 8));
        xmin = fmin(xmin, __shfl_xor_sync(0xffffffffu, xmin, o, 8));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o, 8));
        ymin = fmin(ymin, __shfl_xor_sync(0xffffffffu, ymin, o, 8));
        ymax = fmax(ymax, __shfl_xor_sync(0xffffffffu, ymax, o, 8));
        front |= __shfl_xor_sync(0xffffffffu, front, o, 8);
    }
    if (!active) return -1;
    const double Wd = c.width, Hd = c.height;
    const bool visible = front && xmax > -0.5 && xmin < Wd - 0.5 && ymax > -0.5 && ymin < Hd - 0.5;
    const float* ce = S.block_cell + 4 * (long long)b;
    const bool inside = cp0 >= (double)ce[0] && cp0 < (double)ce[1] && cp1 >= (double)ce[2] && cp1 < (double)ce[3];
    if (!visible && !inside) return -1;
    const double dmin = sqrt(e2);
    int lv = dmin < d1 ? 0 : (dmin < d2 ? 1 : 2);
    if (lv > S.n_levels - 1) lv = S.n_levels - 1;
    return lv;
}

// The same decision in FP32 with a bound on each decided quantity's distance from its FP64
// value, for the groups where every decision is farther from its threshold than that bound (the
// FP64 evaluation above decides the rest; *amb is set for the whole group).  Bounds, u = 2^-24
// (this file is compiled without multiply-add contraction, one rounding per operation):
//   e = p - c and e2 = (e0^2 + e1^2) + e2^2 have relative error <= 8u (positive terms);
//   t = ((R0 p0 + R1 p1) + R2 p2) + t0 per row: <= 5u S, S = the sum of the terms' magnitudes
//   (three product and three sum roundings; the FP64 products of FP32 values are exact);
//   q = tx / tz: <= (5u Sx + |q| 5u Sz) / (tz - 5u Sz) + u |q|; u_pix = fx q + cx adds
//   u |fx q| + u |u_pix|; every screen bound is doubled before it is compared.
__device__ int lod_level8_f32(const cgs_scene& S, int b, const cgs_camera& c, float near_z, double d1, double d2,
                              bool* amb)
{
    const float U = 5.9604645e-8f;
    const int k = threadIdx.x & 7;
    // every value of the block read up front (no load waits on another): its level-0 count,
    // this lane's corner and the ground cell
    const bool inrange = b >= 0 && b < S.n_blocks;
    const long long bq = inrange ? b : 0;
    const long long cnt0 = inrange ? S.level_count[bq * S.n_levels] : 0;
    float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, ce[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (inrange && S.block_aabb) {
        const float* bb = S.block_aabb + 6 * bq;
        p0 = bb[(k & 1) ? 3 : 0];
        p1 = bb[(k & 2) ? 4 : 1];
        p2 = bb[(k & 4) ? 5 : 2];
    }
    if (inrange && S.block_cell) {
        const float* cp = S.block_cell + 4 * bq;
        ce[0] = cp[0]; ce[1] = cp[1]; ce[2] = cp[2]; ce[3] = cp[3];
    }
    const bool active = inrange && cnt0 > 0;
    float e2 = INFINITY, xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY, exu = 0.0f, eyv = 0.0f;
    int front = 0, unsure = 0;
    if (active) {
        const float e0 = p0 - c.campos[0], ee1 = p1 - c.campos[1], ee2 = p2 - c.campos[2];
        e2 = (e0 * e0 + ee1 * ee1) + ee2 * ee2;
        const float tx = ((c.R[0] * p0 + c.R[1] * p1) + c.R[2] * p2) + c.t[0];
        const float ty = ((c.R[3] * p0 + c.R[4] * p1) + c.R[5] * p2) + c.t[1];
        const float tz = ((c.R[6] * p0 + c.R[7] * p1) + c.R[8] * p2) + c.t[2];
        const float ex = 5.0f * U * (((fabsf(c.R[0] * p0) + fabsf(c.R[1] * p1)) + fabsf(c.R[2] * p2)) + fabsf(c.t[0]));
        const float ey = 5.0f * U * (((fabsf(c.R[3] * p0) + fabsf(c.R[4] * p1)) + fabsf(c.R[5] * p2)) + fabsf(c.t[1]));
        const float ez = 5.0f * U * (((fabsf(c.R[6] * p0) + fabsf(c.R[7] * p1)) + fabsf(c.R[8] * p2)) + fabsf(c.t[2]));
        if (tz - ez > near_z) {
            front = 1;
            const float q = tx / tz, r = ty / tz;
            const float dq = (ex + fabsf(q) * ez) / (tz - ez) + U * fabsf(q);
            const float dr = (ey + fabsf(r) * ez) / (tz - ez) + U * fabsf(r);
            const float u = c.fx * q + c.cx, v = c.fy * r + c.cy;
            exu = 2.0f * (fabsf(c.fx) * dq + U * fabsf(c.fx * q) + U * fabsf(u));
            eyv = 2.0f * (fabsf(c.fy) * dr + U * fabsf(c.fy * r) + U * fabsf(v));
            xmin = xmax = u;
            ymin = ymax = v;
        } else if (!(tz + ez <= near_z)) {
            unsure = 1;  // the near-plane decision (or a NaN)
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        e2 = fminf(e2, __shfl_xor_sync(0xffffffffu, e2, o, 8));
        xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, o, 8));
        xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o, 8));
        ymin = fminf(ymin, __shfl_xor_sync(0xffffffffu, ymin, o, 8));
        ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o, 8));
        exu = fmaxf(exu, __shfl_xor_sync(0xffffffffu, exu, o, 8));
        eyv = fmaxf(eyv, __shfl_xor_sync(0xffffffffu, eyv, o, 8));
        front |= __shfl_xor_sync(0xffffffffu, front, o, 8);
        unsure |= __shfl_xor_sync(0xffffffffu, unsure, o, 8);
    }
    *amb = false;
    if (!active) return -1;
    if (unsure) {
        *amb = true;
        return -1;
    }
    // three-valued comparisons: 1 certainly true, 0 certainly false, -1 too close to tell
    auto gt = [](float x, float err, float t) { return x - err > t ? 1 : (x + err <= t ? 0 : -1); };
    auto lt = [](float x, float err, float t) { return x + err < t ? 1 : (x - err >= t ? 0 : -1); };
    const float Wd = (float)c.width, Hd = (float)c.height;
    int vis = 0;
    if (front) {
        const int t4[4] = {gt(xmax, exu, -0.5f), lt(xmin, exu, Wd - 0.5f), gt(ymax, eyv, -0.5f),
                           lt(ymin, eyv, Hd - 0.5f)};
        vis = 1;
        for (int i = 0; i < 4; i++) {
            if (t4[i] == 0) { vis = 0; break; }
            if (t4[i] < 0) vis = -1;
        }
    }
    const bool inside = c.campos[0] >= ce[0] && c.campos[0] < ce[1] && c.campos[1] >= ce[2] && c.campos[1] < ce[3];
    if (!inside) {
        if (vis < 0) { *amb = true; return -1; }
        if (vis == 0) return -1;
    }
    // level: dmin = sqrt(e2min) against d1, d2 (FP64 sqrt is monotone and correctly rounded)
    const double e2d = (double)e2;
    auto less = [&](double d) {
        const double t = d * d;
        if (e2d * (1.0 + 16.0 * (double)U) < t * (1.0 - 1e-12)) return 1;
        if (e2d * (1.0 - 16.0 * (double)U) > t * (1.0 + 1e-12)) return 0;
        return -1;
    };
    int lv;
    const int c1 = less(d1);
    if (c1 < 0) { *amb = true; return -1; }
    if (c1) {
        lv = 0;
    } else {
        const int c2 = less(d2);
        if (c2 < 0) { *amb = true; return -1; }
        lv = c2 ? 1 : 2;
    }
    if (lv > S.n_levels - 1) lv = S.n_levels - 1;
    return lv;
}

// Level of block b for the calling 8-lane group: FP32 where it is certain, FP64 otherwise (all
// lanes of the warp must call it).
__device__ int lod_level8_fast(const cgs_scene& S, int b, const cgs_camera& c, double near_z, double d1, double d2)
{
    bool amb = false;
    const int l = lod_level8_f32(S, b, c, (float)near_z, d1, d2, &amb);
    if (__any_sync(0xffffffffu, amb)) return lod_level8(S, b, c, near_z, d1, d2);
    return l;
}

__global__ void k_lod_levels(cgs_scene S, const cgs_camera* __restrict__ cams, int n_views, cgs_config cfg,
                             int8_t* levels)
{
    const int v = blockIdx.x;
    if (v >= n_views) return;
    const cgs_camera c = cams[v];
    const int groups = blockDim.x >> 3;
    for (int b0 = 0; b0 < S.n_blocks; b0 += groups) {
        const int b = b0 + (threadIdx.x >> 3);
        const int l = lod_level8_fast(S, b < S.n_blocks ? b : -1, c, (double)cfg.near_z, cfg.lod_dist[0], cfg.lod_dist[1]);
        if (b < S.n_blocks && (threadIdx.x & 7) == 0) levels[(long long)v * S.n_blocks + b] = (int8_t)l;
    }
}

// Per view, in two phases.  Phase 1, spread over ceil(n_blocks / SEL_BLOCKS) CTAs per view so
// that the FP64 corner arithmetic of many blocks runs on many SMs: the level of each block
// (given, one training block, or LoD).  Phase 2, in the last CTA of the view to finish phase 1:
// the ordered list of selected segments (fusion by concatenation, Sec. 3.3.2) and its prefix
// counts; the last view to finish also writes the prefix of the per-view counts (the views'
// bases in the flattened selected list).
constexpr int SEL_BLOCKS = 8;                // blocks per CTA in phase 1 (one 8-lane group each)
constexpr int SEL_THREADS = SEL_BLOCKS * 8;  // 64

__global__ void __launch_bounds__(SEL_THREADS) k_select(Layout L, cgs_scene S, const cgs_camera* __restrict__ cams,
                                                        const int32_t* view_block, const int8_t* levels_in,
                                                        cgs_config cfg)
{
    const int v = blockIdx.y;
    const int NB = S.n_blocks, NL = S.n_levels;
    int8_t* lev = L.levels + (long long)v * NB;
    const int b0 = blockIdx.x * SEL_BLOCKS;
    // this CTA's blocks: level, and the chosen level's count and offset (a view of at most
    // SEL_BLOCKS blocks is handled by one CTA, whose second phase reads them from here)
    __shared__ int s_lv[SEL_BLOCKS];
    __shared__ long long s_cnt[SEL_BLOCKS], s_off[SEL_BLOCKS];
    auto keep = [&](int b, int l) {
        long long cnt = 0, off = 0;
        if (l >= 0) {
            cnt = S.level_count[(long long)b * NL + l];
            off = S.level_offset[(long long)b * NL + l];
            if (cnt <= 0) l = -1;
        }
        lev[b] = (int8_t)l;
        s_lv[b - b0] = l;
        s_cnt[b - b0] = cnt;
        s_off[b - b0] = off;
    };
    if (levels_in || view_block) {
        const int b = b0 + (int)threadIdx.x;
        if (threadIdx.x < SEL_BLOCKS && b < NB) {
            int l;
            if (levels_in) {
                l = levels_in[(long long)v * NB + b];
                if (l >= NL) l = NL - 1;
                if (l < 0) l = -1;
            } else {
                l = (b == view_block[v]) ? 0 : -1;
            }
            keep(b, l);
        }
    } else if (L.lod_mode == CGS_LOD_POINT) {
        // point-wise baseline: every non-empty block at its finest level; k_project applies the
        // per-Gaussian distance test
        const int b = b0 + (int)threadIdx.x;
        if (threadIdx.x < SEL_BLOCKS && b < NB) keep(b, 0);
    } else {
        const cgs_camera c = cams[v];
        const int b = b0 + (int)(threadIdx.x >> 3);
        // the counts and offsets of the three levels the LoD can choose, fetched together with
        // the block's bounds instead of after the level is known
        const bool lead = b < NB && (threadIdx.x & 7) == 0;
        long long pc[3] = {0, 0, 0}, po[3] = {0, 0, 0};
        if (lead) {
#pragma unroll
            for (int q = 0; q < 3; q++) {
                if (q < NL) {
                    pc[q] = S.level_count[(long long)b * NL + q];
                    po[q] = S.level_offset[(long long)b * NL + q];
                }
            }
        }
        int l = lod_level8_fast(S, b < NB ? b : -1, c, (double)cfg.near_z, cfg.lod_dist[0], cfg.lod_dist[1]);
        if (lead) {
            // l <= min(2, NL - 1)
            const long long cnt = l >= 0 ? (l == 0 ? pc[0] : (l == 1 ? pc[1] : pc[2])) : 0;
            const long long off = l >= 0 ? (l == 0 ? po[0] : (l == 1 ? po[1] : po[2])) : 0;
            if (l >= 0 && cnt <= 0) l = -1;
            lev[b] = (int8_t)l;
            s_lv[b - b0] = l;
            s_cnt[b - b0] = l >= 0 ? cnt : 0;
            s_off[b - b0] = l >= 0 ? off : 0;
        }
    }
    const bool one_cta = gridDim.x == 1;
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        // a view handled by one CTA needs no hand-off
        if (gridDim.x > 1) {
            __threadfence();
            s_last = atomicAdd(&L.sel_done[v], 1u) == gridDim.x - 1u;
        } else {
            s_last = true;
        }
    }
    __syncthreads();
    if (!s_last) return;
    if (!one_cta) __threadfence();
    // phase 2: the ordered segment list, one CTA-wide exclusive scan per chunk of blocks of the
    // packed pair (selected count << 0 | Gaussian count << SEG_BITS); the levels written by the
    // other CTAs are read past L1
    constexpr int SEG_BITS = 20;  // n_blocks < 2^20
    __shared__ unsigned long long wb[33];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    uint32_t* sb = L.seg_base + (long long)v * (NB + 1);
    long long* so = L.seg_off + (long long)v * NB;
    for (int c0 = 0; c0 < NB; c0 += blockDim.x) {
        const int b = c0 + threadIdx.x;
        const int l = b < NB ? (one_cta ? s_lv[b] : (int)__ldcg(lev + b)) : -1;
        const unsigned long long cnt =
            l >= 0 ? (unsigned long long)(one_cta ? s_cnt[b] : S.level_count[(long long)b * NL + l]) : 0ull;
        const unsigned long long x = l >= 0 ? (1ull | (cnt << SEG_BITS)) : 0ull;
        unsigned long long tot;
        const unsigned long long ex = s_carry + block_exclusive_scan<unsigned long long>(x, wb, &tot);
        if (l >= 0) {
            const int sidx = (int)(ex & ((1ull << SEG_BITS) - 1));
            const unsigned long long acc = ex >> SEG_BITS;
            so[sidx] = one_cta ? s_off[b] : S.level_offset[(long long)b * NL + l];
            L.seg_blk[(long long)v * NB + sidx] = b;
            sb[sidx] = (uint32_t)(acc < 0xffffffffull ? acc : 0xffffffffull);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int ns = (int)(s_carry & ((1ull << SEG_BITS) - 1));
        const unsigned long long acc = s_carry >> SEG_BITS;
        sb[ns] = (uint32_t)(acc < 0xffffffffull ? acc : 0xffffffffull);
        L.n_seg[v] = (uint32_t)ns;
        L.view_cnt[v] = (uint32_t)(acc < 0xffffffffull ? acc : 0xffffffffull);
        // the last view to get here writes the per-view prefix
        if (L.V > 1) {
            __threadfence();
            s_last = atomicAdd(&L.hdr->ctr[CTR_SELECT], 1u) == (uint32_t)L.V - 1u;
        } else {
            s_last = true;
        }
    }
    __syncthreads();
    if (!s_last) return;
    const int V = L.V;
    if (V == 1) {  // one view: its count is the total
        if (threadIdx.x == 0) {
            const unsigned long long total = s_carry >> SEG_BITS;
            L.view_base[0] = 0u;
            L.view_base[1] = (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull);
            L.hdr->n_sel_raw = total;
            const unsigned long long cap = (unsigned long long)L.n_cap;
            L.hdr->n_sel = (uint32_t)(total < cap ? total : cap);
            if (total > cap) latch(L.hdr, ST_CAPACITY);
        }
        return;
    }
    __threadfence();
    // exclusive prefix of the per-view counts; total capped at the frame capacity
    const int per = (V + blockDim.x - 1) / blockDim.x;
    const int v0 = threadIdx.x * per;
    const volatile uint32_t* vc = L.view_cnt;
    unsigned long long local = 0;
    for (int w = v0; w < v0 + per && w < V; w++) local += vc[w];
    unsigned long long total;
    unsigned long long run = block_exclusive_scan<unsigned long long>(local, wb, &total);
    for (int w = v0; w < v0 + per && w < V; w++) {
        L.view_base[w] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
        run += vc[w];
    }
    if (threadIdx.x == 0) {
        L.view_base[V] = (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull);
        L.hdr->n_sel_raw = total;
        unsigned long long cap = (unsigned long long)L.n_cap;
        L.hdr->n_sel = (uint32_t)(total < cap ? total : cap);
        if (total > cap) latch(L.hdr, ST_CAPACITY);
    }
}

// ---------------------------------------------------------------------------------------
// Eq. 7 MAD bounds by exact radix selection.  One CTA per (block, axis).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t f2o(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(uint32_t o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Selects the keys of ranks r0 and r1 (0-based, ascending) among m keys produced by key(k).
// KEY is uint32_t or unsigned long long; runs in all threads of the CTA.
template <typename KEY, typename F>
__device__ void radix_select2(long long m, F key, unsigned long long r0, unsigned long long r1, KEY* out0, KEY* out1)
{
    constexpr int KBITS = sizeof(KEY) * 8;
    __shared__ uint32_t h0[256], h1[256];
    __shared__ KEY s_pre[2], s_mask;
    __shared__ unsigned long long s_rank[2];
    if (threadIdx.x == 0) { s_pre[0] = s_pre[1] = 0; s_mask = 0; s_rank[0] = r0; s_rank[1] = r1; }
    __syncthreads();
    for (int shift = KBITS - 8; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) { h0[i] = 0; h1[i] = 0; }
        __syncthreads();
        const KEY mask = s_mask, p0 = s_pre[0], p1 = s_pre[1];
        for (long long k = threadIdx.x; k < m; k += blockDim.x) {
            const KEY x = key(k);
            const uint32_t d = (uint32_t)(x >> shift) & 255u;
            if ((x & mask) == p0) atomicAdd(&h0[d], 1u);
            if ((x & mask) == p1) atomicAdd(&h1[d], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            uint32_t* h = threadIdx.x == 0 ? h0 : h1;
            unsigned long long r = s_rank[threadIdx.x], cum = 0;
            int d = 0;
            for (; d < 255; d++) {
                if (cum + h[d] > r) break;
                cum += h[d];
            }
            s_rank[threadIdx.x] = r - cum;
            s_pre[threadIdx.x] |= (KEY)d << shift;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_mask |= (KEY)255 << shift;
        __syncthreads();
    }
    *out0 = s_pre[0];
    *out1 = s_pre[1];
    __syncthreads();
}

__device__ __forceinline__ float round_down_f(double x)
{
    float f = __double2float_rn(x);
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}
__device__ __forceinline__ float round_up_f(double x)
{
    float f = __double2float_rn(x);
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

__global__ void __launch_bounds__(256) k_block_bounds(cgs_scene S, double n_mad, float* aabb)
{
    const int b = blockIdx.x / 3, a = blockIdx.x % 3;
    const long long off = S.level_offset[(long long)b * S.n_levels];
    const long long m = S.level_count[(long long)b * S.n_levels];
    if (m <= 0) {
        if (threadIdx.x == 0) { aabb[6 * b + a] = 0.0f; aabb[6 * b + 3 + a] = 0.0f; }
        return;
    }
    const float* base = S.mean_opac + 4 * off + a;
    // min and max
    __shared__ float s_mn[32], s_mx[32];
    float mn = INFINITY, mx = -INFINITY;
    for (long long k = threadIdx.x; k < m; k += blockDim.x) {
        const float x = base[4 * k];
        mn = fminf(mn, x);
        mx = fmaxf(mx, x);
    }
    for (int o = 16; o; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) { s_mn[threadIdx.x >> 5] = mn; s_mx[threadIdx.x >> 5] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) { s_mn[0] = fminf(s_mn[0], s_mn[w]); s_mx[0] = fmaxf(s_mx[0], s_mx[w]); }
    }
    __syncthreads();
    const double dmn = (double)s_mn[0], dmx = (double)s_mx[0];
    // median: ranks (m-1)/2 and m/2 of the values
    uint32_t o0, o1;
    radix_select2<uint32_t>(m, [&](long long k) { return f2o(base[4 * k]); }, (unsigned long long)((m - 1) / 2),
                            (unsigned long long)(m / 2), &o0, &o1);
    const double med = ((double)o2f(o0) + (double)o2f(o1)) * 0.5;
    // MAD: the same ranks of |p - median| (non-negative doubles order like their bits)
    unsigned long long a0, a1;
    radix_select2<unsigned long long>(
        m, [&](long long k) { return (unsigned long long)__double_as_longlong(fabs((double)base[4 * k] - med)); },
        (unsigned long long)((m - 1) / 2), (unsigned long long)(m / 2), &a0, &a1);
    const double mad = (__longlong_as_double((long long)a0) + __longlong_as_double((long long)a1)) * 0.5;
    if (threadIdx.x == 0) {
        double lo = med - n_mad * mad, hi = med + n_mad * mad;
        if (dmn > lo) lo = dmn;
        if (dmx < hi) hi = dmx;
        aabb[6 * b + a] = round_down_f(lo);
        aabb[6 * b + 3 + a] = round_up_f(hi);
    }
}

void launch_select(const Layout& L, const cgs_scene& S, const cgs_camera* cams, const int32_t* view_block,
                   const int8_t* levels, const cgs_config& cfg, cudaStream_t st)
{
    const dim3 grid((unsigned)((S.n_blocks + SEL_BLOCKS - 1) / SEL_BLOCKS), (unsigned)L.V);
    k_select<<<grid, SEL_THREADS, 0, st>>>(L, S, cams, view_block, levels, cfg);
}

void launch_lod_levels(const cgs_scene& S, const cgs_config& cfg, const cgs_camera* cams, int n_views,
                       int8_t* levels, cudaStream_t st)
{
    k_lod_levels<<<n_views, 256, 0, st>>>(S, cams, n_views, cfg, levels);
}

void launch_block_bounds(const cgs_scene& S, double n_mad, float* aabb, cudaStream_t st)
{
    k_block_bounds<<<S.n_blocks * 3, 256, 0, st>>>(S, n_mad, aabb);
}

}  // namespace cgs
