// Stage d of the hot path: per-tile front-to-back alpha compositing (Eq. 1, Sec. 3.1) and
// its backward replay (differentiable rendering, Sec. 3.1), plus the L1 loss (Sec. 3.2.3).
//
// One CTA per (view, tile), one thread per pixel.  Each round stages `BATCH` projected
// records of the tile's depth-sorted list in shared memory; a pixel blends with
// alpha = min(0.99, o exp(power)), skips alpha < 1/255 and stops before the entry that
// would take its transmittance below 1e-4.  The CTA leaves as soon as every pixel stopped
// (__syncthreads_count).
#include "common.cuh"

namespace cgs {

// power = -0.5 A' dx^2 - B' dx dy - 0.5 C' dy^2 at a lane's two pixels (px, py0) and
// (px, py1), which share dx, with every rounding step fixed by intrinsics so the forward and
// the backward kernels take identical decisions.
__device__ __forceinline__ void pair_power2(const float4& a, const float4& b, float fpx, float fpy0, float fpy1,
                                            float* pw0, float* pw1, float* dx_out, float* dy0_out, float* dy1_out)
{
    const float dx = __fsub_rn(a.x, fpx), dy0 = __fsub_rn(a.y, fpy0), dy1 = __fsub_rn(a.y, fpy1);
    const float hC = __fmul_rn(-0.5f, b.z);
    const float ax = __fmul_rn(__fmul_rn(__fmul_rn(-0.5f, b.x), dx), dx);  // -A' dx^2 / 2
    const float nbx = __fmul_rn(-b.y, dx);                                  // -B' dx
    *pw0 = __fmaf_rn(__fmul_rn(hC, dy0), dy0, __fmaf_rn(nbx, dy0, ax));
    *pw1 = __fmaf_rn(__fmul_rn(hC, dy1), dy1, __fmaf_rn(nbx, dy1, ax));
    *dx_out = dx;
    *dy0_out = dy0;
    *dy1_out = dy1;
}

// Warp sum of 32 values per lane by halving exchanges: at each step a lane keeps half of its
// values and adds the partner's copy of that half.  On return lane l holds the warp total of
// v[l] (31 shuffles for 32 sums).
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32], int lane)
{
#pragma unroll
    for (int o = 16, n = 16; o >= 1; o >>= 1, n >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < n; k++) {
            const float send = hi ? v[k] : v[k + n];
            const float keep = hi ? v[k + n] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// Threads of a B x B tile: B*B/2, two pixels each.  Warp w covers the 8 x 8 block at
// ((w % (B/8)) * 8, (w / (B/8)) * 8); lane l takes pixels (l & 7, l >> 3) and (l & 7, (l >> 3) + 4).
template <int B>
__device__ __forceinline__ void pixels_of(int tid, int* x, int* y0, int* wx0, int* wy0)
{
    const int w = tid >> 5, lane = tid & 31;
    *wx0 = (w % (B / 8)) * 8;
    *wy0 = (w / (B / 8)) * 8;
    *x = *wx0 + (lane & 7);
    *y0 = *wy0 + (lane >> 3);
}

// Whole-warp skip: true if the Gaussian's 1/255 extent box (record .w lanes) misses the
// warp's 8 x 8 pixel block [bx0, bx0 + 7] x [by0, by0 + 7].  Skipped pairs would all fail
// the alpha >= 1/255 test, so skipping changes no result.
__device__ __forceinline__ bool warp_culled(const float4& a, const float4& b, float bx0, float by0)
{
    const float dx = fmaxf(fmaxf(bx0 - a.x, a.x - (bx0 + 7.0f)), 0.0f);
    const float dy = fmaxf(fmaxf(by0 - a.y, a.y - (by0 + 7.0f)), 0.0f);
    return dx > a.w || dy > b.w;
}

// Minimum over the pixel-centre box [x0, x0 + 7] x [y0, y0 + 7] of the quadratic form
// q(d) = A' dx^2 + 2 B' dx dy + C' dy^2, d = p - (u, v), or 0 if the centre lies inside.
// For a convex q with its minimum outside the box, the box minimum lies on an edge; along an
// edge q is a parabola minimised at the clamped stationary point.
__device__ __forceinline__ float box_min_q(const float4& a, const float4& b, float x0, float y0)
{
    const float dx0 = x0 - a.x, dx1 = x0 + 7.0f - a.x, dy0 = y0 - a.y, dy1 = y0 + 7.0f - a.y;
    if (dx0 <= 0.0f && dx1 >= 0.0f && dy0 <= 0.0f && dy1 >= 0.0f) return 0.0f;
    const float qa = b.x, qb = b.y, qc = b.z;
    float m = INFINITY;
#pragma unroll
    for (int e = 0; e < 2; e++) {
        const float dx = e ? dx1 : dx0;
        const float dy = fminf(fmaxf(-qb * dx / qc, dy0), dy1);
        m = fminf(m, qa * dx * dx + 2.0f * qb * dx * dy + qc * dy * dy);
        const float ey = e ? dy1 : dy0;
        const float ex = fminf(fmaxf(-qb * ey / qa, dx0), dx1);
        m = fminf(m, qa * ex * ex + 2.0f * qb * ex * ey + qc * ey * ey);
    }
    return m;
}

// Bit w set: the Gaussian can pass the 1/255 test at some pixel of warp w's block of the
// tile whose top-left pixel is (tx0, ty0): its extent box meets the block and the block's
// minimum of q is within the slackened threshold t (record c.w; +inf disables the test).
template <int B>
__device__ __forceinline__ uint32_t warp_mask(const float4& a, const float4& b, float t, float tx0, float ty0)
{
    constexpr int NW = B * B / 64;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const float bx0 = tx0 + (float)((w % (B / 8)) * 8), by0 = ty0 + (float)((w / (B / 8)) * 8);
        if (warp_culled(a, b, bx0, by0)) continue;
        if (t < INFINITY && box_min_q(a, b, bx0, by0) > t) continue;
        m |= 1u << w;
    }
    return m;
}

// Forward blend of one entry into one pixel (Eq. 1 with the 3DGS thresholds).  Written
// without branches: a warp runs every step for all its lanes anyway, and the predicated form
// saves the divergence bookkeeping.  A pair that does not blend adds c * 0 (exactly nothing)
// and keeps T and last.
struct FwdPixel {
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0, stop_at = 0xffffffffu;
    bool done = false;
    __device__ __forceinline__ bool blend(float power, float o, const float4& c, uint32_t pos)
    {
        const float alpha = fminf(0.99f, __fmul_rn(o, __expf(power)));
        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, alpha));
        const bool ok = !done && !(power > 0.0f) && !(alpha < 1.0f / 255.0f);
        const bool stop = ok && Tn < 1e-4f;
        const bool use = ok && !stop;
        const float w = use ? alpha * T : 0.0f;
        C0 += c.x * w;
        C1 += c.y * w;
        C2 += c.z * w;
        if (stop) {
            done = true;
            stop_at = pos;
        }
        T = use ? Tn : T;
        last = use ? pos + 1u : last;
        return use;
    }
};

// Forward.  Staging a batch, each loading thread also records which warps its Gaussian can
// reach; each warp then visits only those entries (ballot over 32-entry chunks), in list
// order.  n_contrib and the evaluated-pair count keep the semantics of a walk over the full
// list: entries up to and including the stopping one, or the whole list.
//
// With HITS, every blend is also counted per scene Gaussian: one atomic add per (warp, entry)
// of the number of the warp's pixels that blended it (L.hits, indexed by scene index).
template <int B, int BATCH, bool HITS>
__global__ void __launch_bounds__(B * B / 2, B == 16 ? 8 : 32) k_render_fwd(Layout L, const uint32_t* __restrict__ tval, float bg0,
                                                          float bg1, float bg2, float* __restrict__ image,
                                                          float* __restrict__ final_T, uint32_t* __restrict__ n_contrib)
{
    constexpr int NT = B * B / 2;
    __shared__ float4 s_a[BATCH], s_b[BATCH], s_c[BATCH];
    __shared__ uint32_t s_m[BATCH];
    __shared__ uint32_t s_g[HITS ? BATCH : 1];
    const int v = blockIdx.z;
    const int tile = blockIdx.y * L.tiles_x + blockIdx.x;
    const uint2 rg = reinterpret_cast<const uint2*>(L.ranges)[(size_t)v * L.T + tile];
    int lx, ly, wx0, wy0;
    pixels_of<B>(threadIdx.x, &lx, &ly, &wx0, &wy0);
    const int px = blockIdx.x * B + lx, py0 = blockIdx.y * B + ly, py1 = py0 + 4;
    const bool in0 = px < L.W && py0 < L.H, in1 = px < L.W && py1 < L.H;
    const float fpx = (float)px, fpy0 = (float)py0, fpy1 = (float)py1;
    const float tx0 = (float)(blockIdx.x * B), ty0 = (float)(blockIdx.y * B);
    const int lane = threadIdx.x & 31;
    const uint32_t wbit = 1u << (threadIdx.x >> 5);
    // this warp's contribution words: NW * (start / 32 + tile index) + warp * (len / 32 + 1)
    constexpr int NW = B * B / 64;
    const size_t tg = (size_t)v * L.T + tile;
    uint32_t* cbits = L.cbits + (size_t)NW * (rg.x / 32 + tg) + (size_t)(threadIdx.x >> 5) * ((rg.y - rg.x) / 32 + 1);
    uint32_t steps = 0, useful = 0;  // warp steps visited / with a blend (lane 0 counts)
    FwdPixel p0, p1;
    p0.done = !in0;
    p1.done = !in1;
    for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
        if (__syncthreads_count(p0.done && p1.done) == NT) break;
        for (int i = threadIdx.x; i < BATCH; i += NT) {
            uint32_t m = 0;
            if (start + i < rg.y) {
                const size_t j = tval[start + i];
                const float4 a = L.rec[3 * j], b = L.rec[3 * j + 1], c = L.rec[3 * j + 2];
                s_a[i] = a;
                s_b[i] = b;
                s_c[i] = c;
                m = warp_mask<B>(a, b, c.w, tx0, ty0);
                if (HITS) s_g[i] = L.gidx[j];
            }
            s_m[i] = m;
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)BATCH, rg.y - start);
        for (int c0 = 0; c0 < nb; c0 += 32) {
            if (__all_sync(0xffffffffu, p0.done && p1.done)) break;
            uint32_t bits = __ballot_sync(0xffffffffu, c0 + lane < nb && (s_m[c0 + lane] & wbit));
            const uint32_t s_bits = bits;
            uint32_t word = 0;
            while (bits) {
                const int kk = __ffs(bits) - 1;
                bits &= bits - 1;
                const int k = c0 + kk;
                const float4 a = s_a[k], b = s_b[k], c = s_c[k];
                const uint32_t pos = start - rg.x + (uint32_t)k;
                float pw0, pw1, dx, dy0, dy1;
                pair_power2(a, b, fpx, fpy0, fpy1, &pw0, &pw1, &dx, &dy0, &dy1);
                const bool b0 = p0.blend(pw0, a.z, c, pos);
                const bool b1 = p1.blend(pw1, a.z, c, pos);
                if (__any_sync(0xffffffffu, b0 || b1)) word |= 1u << kk;
                if (HITS) {
                    const int cnt = __popc(__ballot_sync(0xffffffffu, b0)) + __popc(__ballot_sync(0xffffffffu, b1));
                    if (lane == 0 && cnt) atomicAdd(&L.hits[s_g[k]], (uint32_t)cnt);
                }
            }
            if (lane == 0) {
                cbits[(start - rg.x + c0) >> 5] = word;
                steps += (uint32_t)__popc(s_bits);
                useful += (uint32_t)__popc(word);
            }
        }
    }
    const size_t HW = (size_t)L.W * L.H;
    if (in0) {
        const size_t pix = (size_t)py0 * L.W + px;
        image[(3 * (size_t)v + 0) * HW + pix] = p0.C0 + p0.T * bg0;
        image[(3 * (size_t)v + 1) * HW + pix] = p0.C1 + p0.T * bg1;
        image[(3 * (size_t)v + 2) * HW + pix] = p0.C2 + p0.T * bg2;
        final_T[(size_t)v * HW + pix] = p0.T;
        n_contrib[(size_t)v * HW + pix] = p0.last;
    }
    if (in1) {
        const size_t pix = (size_t)py1 * L.W + px;
        image[(3 * (size_t)v + 0) * HW + pix] = p1.C0 + p1.T * bg0;
        image[(3 * (size_t)v + 1) * HW + pix] = p1.C1 + p1.T * bg1;
        image[(3 * (size_t)v + 2) * HW + pix] = p1.C2 + p1.T * bg2;
        final_T[(size_t)v * HW + pix] = p1.T;
        n_contrib[(size_t)v * HW + pix] = p1.last;
    }
    const uint32_t len = rg.y - rg.x;
    const uint32_t visited = (in0 ? (p0.stop_at != 0xffffffffu ? p0.stop_at + 1u : len) : 0u) +
                             (in1 ? (p1.stop_at != 0xffffffffu ? p1.stop_at + 1u : len) : 0u);
    const uint32_t ws = __reduce_add_sync(0xffffffffu, visited);
    if (lane == 0) {
        if (ws) atomicAdd(&L.hdr->pairs_fwd, (unsigned long long)ws);
        if (steps) atomicAdd(&L.hdr->steps_fwd, (unsigned long long)steps);
        if (useful) atomicAdd(&L.hdr->steps_useful, (unsigned long long)useful);
    }
}

// Backward replay of one pixel.  The pixel visits its blended entries from the last one
// (n_contrib) to the first, recovering T before entry i as T_{i+1} / (1 - alpha_i) from the
// final transmittance.  With g = dL/dP (per channel) and S_i = sum_{m > i} alpha_m T_m c_m
// + T_end bg, only the scalar gS = g . S_i is needed:
//   dL/dc_i = g alpha_i T_i,  dL/dalpha_i = T_i (g . c_i) - gS / (1 - alpha_i),
//   alpha = min(0.99, o G), G = exp(power): dalpha/do = G, dalpha/dpower = o G (not clamped).
// With dp = dL/dpower, the accumulated values are
//   m[0..4] = sum dp dx, sum dp dy, sum dp dx^2, sum dp dx dy, sum dp dy^2,
//   m[5] = dL/do, m[6..8] = dL/d(r, g, b),
// from which the per-Gaussian factors of the conic give dL/d(u, v, A', B', C') (flush).
struct BwdPixel {
    float T = 1.0f, gS = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    uint32_t nc = 0;
    // Predicated like the forward: a pair that did not blend leaves T and gS and adds exact
    // zeros (selected, never multiplied, so no inf * 0 reaches the sums).  SET writes the
    // nine sums instead of adding to them (the first pixel of a lane).
    template <bool SET>
    __device__ __forceinline__ bool replay(float power, float dx, float dy, float o, const float4& c, uint32_t lp,
                                           float* m)
    {
        const float G = __expf(power);
        const float og = __fmul_rn(o, G);
        const float alpha = fminf(0.99f, og);
        const bool use = lp < nc && !(power > 0.0f) && !(alpha < 1.0f / 255.0f);
        const float inv = __fdividef(1.0f, 1.0f - alpha);
        const float Tb = T * inv;  // transmittance before this entry
        const float gc = g0 * c.x + g1 * c.y + g2 * c.z;
        const float dal = gc * Tb - gS * inv;
        const float aT = alpha * Tb;
        T = use ? Tb : T;
        gS = use ? gS + aT * gc : gS;
        const float aTu = use ? aT : 0.0f;
        const bool lin = use && !(og > 0.99f);  // the 0.99 clamp passes no gradient
        const float dp = lin ? dal * og : 0.0f;
        const float px = dp * dx, py = dp * dy;
        const float v[9] = {px, py, px * dx, px * dy, py * dy, lin ? dal * G : 0.0f, g0 * aTu, g1 * aTu, g2 * aTu};
#pragma unroll
        for (int i = 0; i < 9; i++) m[i] = SET ? v[i] : m[i] + v[i];
        return use;
    }
};

// Backward.  A warp visits exactly the entries that blended into at least one of its pixels
// in the forward (the forward's contribution bits), three at a time: the 27 sums of the
// three entries over the warp's 64 pixels come out of one transpose reduction (lane l holds
// sum l), are added in shared memory per entry, turned into dL/d(u, v, conic, o, rgb) with
// the entry's conic, and added once per (tile, Gaussian) to the global accumulator.
template <int B, int BATCH>
__global__ void __launch_bounds__(B * B / 2, B == 16 ? 6 : 24) k_render_bwd(Layout L, const uint32_t* __restrict__ tval, float bg0,
                                                          float bg1, float bg2, const float* __restrict__ dL_dimg,
                                                          const float* __restrict__ final_T,
                                                          const uint32_t* __restrict__ n_contrib)
{
    constexpr int NT = B * B / 2;
    constexpr int NW = B * B / 64;
    __shared__ float4 s_a[BATCH], s_b[BATCH], s_c[BATCH];
    __shared__ uint32_t s_j[BATCH];
    __shared__ float s_g[BATCH][9];
    __shared__ uint32_t s_maxnc;
    const int v = blockIdx.z;
    const int tile = blockIdx.y * L.tiles_x + blockIdx.x;
    const uint2 rg = reinterpret_cast<const uint2*>(L.ranges)[(size_t)v * L.T + tile];
    int lx, ly, wx0, wy0;
    pixels_of<B>(threadIdx.x, &lx, &ly, &wx0, &wy0);
    const int px = blockIdx.x * B + lx, py0 = blockIdx.y * B + ly, py1 = py0 + 4;
    const bool in0 = px < L.W && py0 < L.H, in1 = px < L.W && py1 < L.H;
    const float fpx = (float)px, fpy0 = (float)py0, fpy1 = (float)py1;
    const int lane = threadIdx.x & 31;
    const size_t tg = (size_t)v * L.T + tile;
    const uint32_t* cbits =
        L.cbits + (size_t)NW * (rg.x / 32 + tg) + (size_t)(threadIdx.x >> 5) * ((rg.y - rg.x) / 32 + 1);
    const size_t HW = (size_t)L.W * L.H;
    BwdPixel q0, q1;
    if (in0) {
        const size_t pix = (size_t)py0 * L.W + px;
        q0.T = final_T[(size_t)v * HW + pix];
        q0.nc = n_contrib[(size_t)v * HW + pix];
        q0.g0 = dL_dimg[(3 * (size_t)v + 0) * HW + pix];
        q0.g1 = dL_dimg[(3 * (size_t)v + 1) * HW + pix];
        q0.g2 = dL_dimg[(3 * (size_t)v + 2) * HW + pix];
    }
    if (in1) {
        const size_t pix = (size_t)py1 * L.W + px;
        q1.T = final_T[(size_t)v * HW + pix];
        q1.nc = n_contrib[(size_t)v * HW + pix];
        q1.g0 = dL_dimg[(3 * (size_t)v + 0) * HW + pix];
        q1.g1 = dL_dimg[(3 * (size_t)v + 1) * HW + pix];
        q1.g2 = dL_dimg[(3 * (size_t)v + 2) * HW + pix];
    }
    q0.gS = q0.T * (q0.g0 * bg0 + q0.g1 * bg1 + q0.g2 * bg2);
    q1.gS = q1.T * (q1.g0 * bg0 + q1.g1 * bg1 + q1.g2 * bg2);
    if (threadIdx.x == 0) s_maxnc = 0;
    __syncthreads();
    const uint32_t mnc = max(q0.nc, q1.nc);
    if (mnc) atomicMax(&s_maxnc, mnc);
    __syncthreads();
    const long long first = rg.x;
    // n_contrib never exceeds the tile's list length; clamp so a mismatched buffer cannot
    // move the replay outside this tile's entries
    const long long end = (first + s_maxnc) < (long long)rg.y ? (first + s_maxnc) : (long long)rg.y;
    // the forward wrote this warp's contribution words up to its last blended position
    uint32_t wmax = mnc;
#pragma unroll
    for (int o = 16; o; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    uint32_t pairs = 0;
    // batches at list positions that are multiples of BATCH (as in the forward), last first,
    // so contribution words line up with 32-entry chunks
    for (long long bi = (end - first - 1) / BATCH; end > first && bi >= 0; bi--) {
        const long long bs = first + bi * BATCH;
        const long long be = (bs + BATCH) < end ? (bs + BATCH) : end;
        const int nb = (int)(be - bs);
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += NT) {
            const uint32_t j = tval[bs + i];
            s_j[i] = j;
            s_a[i] = L.rec[3 * (size_t)j];
            s_b[i] = L.rec[3 * (size_t)j + 1];
            s_c[i] = L.rec[3 * (size_t)j + 2];
        }
        for (int i = threadIdx.x; i < 9 * BATCH; i += NT) (&s_g[0][0])[i] = 0.0f;
        __syncthreads();
        const int kmax = (int)min((long long)nb, (long long)wmax - (bs - first));  // entries k < kmax
        for (int c0 = ((kmax - 1) & ~31); kmax > 0 && c0 >= 0; c0 -= 32) {
            const int avail = kmax - c0;
            uint32_t bits = cbits[(uint32_t)(bs - first + c0) >> 5];
            if (avail < 32) bits &= (1u << avail) - 1u;
            while (bits) {
                // up to three entries, in descending list order
                int ks[3];
#pragma unroll
                for (int e = 0; e < 3; e++) {
                    if (bits) {
                        const int hb = 31 - __clz(bits);
                        bits &= ~(1u << hb);
                        ks[e] = c0 + hb;
                    } else {
                        ks[e] = -1;
                    }
                }
                float acc[32];
#pragma unroll
                for (int i = 27; i < 32; i++) acc[i] = 0.0f;
#pragma unroll
                for (int e = 0; e < 3; e++) {
                    if (ks[e] < 0) {
#pragma unroll
                        for (int i = 0; i < 9; i++) acc[9 * e + i] = 0.0f;
                        continue;
                    }
                    const int k = ks[e];
                    const float4 a = s_a[k], b = s_b[k], c = s_c[k];
                    const uint32_t lp = (uint32_t)(bs + k - first);
                    float pw0, pw1, dx, dy0, dy1;
                    pair_power2(a, b, fpx, fpy0, fpy1, &pw0, &pw1, &dx, &dy0, &dy1);
                    pairs += (uint32_t)q0.replay<true>(pw0, dx, dy0, a.z, c, lp, acc + 9 * e);
                    pairs += (uint32_t)q1.replay<false>(pw1, dx, dy1, a.z, c, lp, acc + 9 * e);
                }
                const float tot = warp_transpose_sum32(acc, lane);
                if (lane < 27) {
                    const int e = lane / 9, comp = lane - 9 * e;
                    const int k = e == 0 ? ks[0] : (e == 1 ? ks[1] : ks[2]);
                    if (k >= 0 && tot != 0.0f) atomicAdd(&s_g[k][comp], tot);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += NT) {
            float* dst = reinterpret_cast<float*>(L.gs) + 12 * (size_t)s_j[i];
            const float4 cn = s_b[i];  // conic A', B', C'
            const float mx = s_g[i][0], my = s_g[i][1];
            float gsc[9];
            gsc[0] = -(cn.x * mx + cn.y * my);  // dL/du
            gsc[1] = -(cn.z * my + cn.y * mx);  // dL/dv
            gsc[2] = -0.5f * s_g[i][2];         // dL/dA'
            gsc[3] = -s_g[i][3];                // dL/dB'
            gsc[4] = -0.5f * s_g[i][4];         // dL/dC'
#pragma unroll
            for (int c = 5; c < 9; c++) gsc[c] = s_g[i][c];
#pragma unroll
            for (int c = 0; c < 9; c++)
                if (gsc[c] != 0.0f) atomicAdd(dst + c, gsc[c]);
        }
    }
    const uint32_t ws = __reduce_add_sync(0xffffffffu, pairs);
    if (lane == 0 && ws) atomicAdd(&L.hdr->pairs_bwd, (unsigned long long)ws);
}

template <int B, int BATCH>
static void fwd_launch(const Layout& L, const uint32_t* tval, const cgs_config& c, float* img, float* T, uint32_t* nc,
                       cudaStream_t st)
{
    dim3 grid(L.tiles_x, L.tiles_y, L.V);
    if (L.hits)
        k_render_fwd<B, BATCH, true><<<grid, B * B / 2, 0, st>>>(L, tval, c.bg[0], c.bg[1], c.bg[2], img, T, nc);
    else
        k_render_fwd<B, BATCH, false><<<grid, B * B / 2, 0, st>>>(L, tval, c.bg[0], c.bg[1], c.bg[2], img, T, nc);
}
template <int B, int BATCH>
static void bwd_launch(const Layout& L, const uint32_t* tval, const cgs_config& c, const float* dimg, const float* T,
                       const uint32_t* nc, cudaStream_t st)
{
    dim3 grid(L.tiles_x, L.tiles_y, L.V);
    k_render_bwd<B, BATCH><<<grid, B * B / 2, 0, st>>>(L, tval, c.bg[0], c.bg[1], c.bg[2], dimg, T, nc);
}

bool launch_render_fwd(const Layout& L, const cgs_config& c, float* img, float* T, uint32_t* nc, cudaStream_t st)
{
    const uint32_t* tv = L.tval;
    if (L.B == 16) {
        switch (c.batch) {
            case 32: fwd_launch<16, 32>(L, tv, c, img, T, nc, st); return true;
            case 64: fwd_launch<16, 64>(L, tv, c, img, T, nc, st); return true;
            case 128: fwd_launch<16, 128>(L, tv, c, img, T, nc, st); return true;
            case 256: fwd_launch<16, 256>(L, tv, c, img, T, nc, st); return true;
        }
    } else if (L.B == 8) {
        switch (c.batch) {
            case 32: fwd_launch<8, 32>(L, tv, c, img, T, nc, st); return true;
            case 64: fwd_launch<8, 64>(L, tv, c, img, T, nc, st); return true;
        }
    }
    return false;
}

bool launch_render_bwd(const Layout& L, const cgs_config& c, const float* dimg, const float* T, const uint32_t* nc,
                       cudaStream_t st)
{
    const uint32_t* tv = L.tval;
    if (L.B == 16) {
        switch (c.batch) {
            case 32: bwd_launch<16, 32>(L, tv, c, dimg, T, nc, st); return true;
            case 64: bwd_launch<16, 64>(L, tv, c, dimg, T, nc, st); return true;
            case 128: bwd_launch<16, 128>(L, tv, c, dimg, T, nc, st); return true;
            case 256: bwd_launch<16, 256>(L, tv, c, dimg, T, nc, st); return true;
        }
    } else if (L.B == 8) {
        switch (c.batch) {
            case 32: bwd_launch<8, 32>(L, tv, c, dimg, T, nc, st); return true;
            case 64: bwd_launch<8, 64>(L, tv, c, dimg, T, nc, st); return true;
        }
    }
    return false;
}

// L1 loss: loss += mean |img - target|, grad = sign(img - target) / count.  The partial
// sums are reduced per CTA, so the loss takes one atomic per CTA.
// Target value of an FP32 target, or of an 8-bit one (channel value t stands for t / 255,
// correctly rounded: a 256-entry table of __fdiv_rn(t, 255) per CTA).
template <typename TT>
struct TargetMap;
template <>
struct TargetMap<float> {
    __device__ __forceinline__ void init() {}
    __device__ __forceinline__ float operator()(float t) const { return t; }
};
template <>
struct TargetMap<uint8_t> {
    float* tab;
    __device__ __forceinline__ void init()
    {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) tab[i] = __fdiv_rn((float)i, 255.0f);
        __syncthreads();
    }
    __device__ __forceinline__ float operator()(uint8_t t) const { return tab[t]; }
};

template <typename TT>
__device__ __forceinline__ float l1_term(float x, TT t, const TargetMap<TT>& map, float inv, float* g)
{
    const float d = x - map(t);
    *g = d > 0.0f ? inv : (d < 0.0f ? -inv : 0.0f);
    return fabsf(d);
}

// With VEC (all three arrays aligned for it), four values per thread (16-byte image and
// gradient accesses) over the bulk, then a tail; otherwise one value per thread.
template <typename TT, bool VEC>
__global__ void __launch_bounds__(256) k_l1(const float* __restrict__ img, const TT* __restrict__ tgt, long long n,
                                            float* loss, float* __restrict__ grad)
{
    __shared__ float s_w[8];
    __shared__ float s_tab[256];
    TargetMap<TT> map;
    if constexpr (sizeof(TT) == 1) map.tab = s_tab;
    map.init();
    const float inv = 1.0f / (float)n;
    float acc = 0.0f;
    const long long n4 = VEC ? n / 4 : 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const float4* img4 = reinterpret_cast<const float4*>(img);
    float4* grad4 = reinterpret_cast<float4*>(grad);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 x = img4[i];
        TT t[4];
        if constexpr (sizeof(TT) == 1) {
            const uchar4 u = reinterpret_cast<const uchar4*>(tgt)[i];
            t[0] = u.x; t[1] = u.y; t[2] = u.z; t[3] = u.w;
        } else {
            const float4 u = reinterpret_cast<const float4*>(tgt)[i];
            t[0] = u.x; t[1] = u.y; t[2] = u.z; t[3] = u.w;
        }
        float4 g;
        acc += l1_term(x.x, t[0], map, inv, &g.x);
        acc += l1_term(x.y, t[1], map, inv, &g.y);
        acc += l1_term(x.z, t[2], map, inv, &g.z);
        acc += l1_term(x.w, t[3], map, inv, &g.w);
        grad4[i] = g;
    }
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        acc += l1_term(img[i], tgt[i], map, inv, &grad[i]);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_w[w];
        if (t != 0.0f) atomicAdd(loss, t * inv);
    }
}

template <typename TT>
static void l1_launch(const float* img, const TT* tgt, long long n, float* loss, float* grad, int n_sm, cudaStream_t st)
{
    const bool vec = ((uintptr_t)img % 16 == 0) && ((uintptr_t)grad % 16 == 0) && ((uintptr_t)tgt % (4 * sizeof(TT)) == 0);
    long long g = ((vec ? n / 4 : n) + 255) / 256;
    if (g > (long long)n_sm * 8) g = (long long)n_sm * 8;
    if (g < 1) g = 1;
    if (vec) k_l1<TT, true><<<(unsigned)g, 256, 0, st>>>(img, tgt, n, loss, grad);
    else k_l1<TT, false><<<(unsigned)g, 256, 0, st>>>(img, tgt, n, loss, grad);
}

void launch_l1(const float* img, const float* tgt, long long n, float* loss, float* grad, int n_sm, cudaStream_t st)
{
    l1_launch<float>(img, tgt, n, loss, grad, n_sm, st);
}

void launch_l1_u8(const float* img, const uint8_t* tgt, long long n, float* loss, float* grad, int n_sm,
                  cudaStream_t st)
{
    l1_launch<uint8_t>(img, tgt, n, loss, grad, n_sm, st);
}

}  // namespace cgs
