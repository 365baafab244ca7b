// Forward projection of every selected Gaussian (stage b of the hot path): Eq. 1's proj,
// SH colour, screen radius and tile rectangle.  Compiled with -fmad=false so the key path
// is evaluated exactly in the order proj_math.cuh writes it.
#include "proj_math.cuh"

namespace cgs {

// Conservative half-extents (pixels) of the region where alpha = min(0.99, o exp(-q/2)) can
// reach 1/255, i.e. q <= t = 2 ln(255 o).  Since q(d) >= dx^2 / Sigma_xx for a positive
// definite Sigma, |dx| > sqrt(t Sigma_xx) implies alpha < 1/255 (likewise for y).  The
// threshold and extents get relative and absolute slack far above FP32 rounding of q; for
// strongly correlated 2D covariances (rho^2 > 0.99), where the rounding of q is not bounded
// by that slack, the extent is infinite (never culled).  Opacity with o * 255 < 1 can never
// pass the test: extent -1 (always culled); o * 255 == 1 can, at power 0 exactly.
// *tq receives the slackened threshold t itself (for the exact ellipse test of the
// compositing kernels), or +inf when no culling is safe.
__device__ __forceinline__ void cull_extent(float o, float A, float B, float C, float* ex, float* ey, float* tq)
{
    if (!(o * 255.0f >= 1.0f)) { *ex = -1.0f; *ey = -1.0f; *tq = -1.0f; return; }
    if (B * B > 0.99f * A * C) { *ex = INFINITY; *ey = INFINITY; *tq = INFINITY; return; }
    const float t = 2.0f * logf(255.0f * o) * 1.002f + 0.002f;
    *ex = sqrtf(t * A) * 1.001f + 0.01f;
    *ey = sqrtf(t * C) * 1.001f + 0.01f;
    *tq = t;
}

// Conservative test that a Gaussian (camera-space centre t, largest absolute scale sm) cannot
// touch the view's image: its tile rect would be empty.  The 2D covariance is
// J W Sigma3D W^T J^T + 0.3 I with Sigma3D's eigenvalues s_k^2, so its largest eigenvalue is
// at most |J|_F^2 max s_k^2 + 0.3; the radius of the exact path, ceil(3 sqrt(lam1)) with
// lam1 <= that bound + 0.32 (the 0.1 floor of the discriminant), is covered by rb with 1% and
// 2-pixel slack.  The test multiplies by one reciprocal of tz instead of dividing: its error
// and FP32 rounding, a few units in the last place, lie far inside that slack.  True only when
// the exact path's rect is certainly empty (a NaN anywhere keeps the Gaussian).
__device__ __forceinline__ bool surely_off_screen(float sm, const cgs_camera& c, float tx, float ty, float tz, int W,
                                                  int H)
{
    const float itz = __frcp_rn(tz);
    const float limx = 1.3f * ((0.5f * (float)c.width) / c.fx), limy = 1.3f * ((0.5f * (float)c.height) / c.fy);
    const float xzc = fminf(fmaxf(tx * itz, -limx), limx), yzc = fminf(fmaxf(ty * itz, -limy), limy);
    const float j00 = c.fx * itz, j11 = c.fy * itz, j02 = j00 * xzc, j12 = j11 * yzc;
    const float jn = j00 * j00 + j02 * j02 + j11 * j11 + j12 * j12;
    const float rb = 3.0f * sqrtf((jn * sm * sm + 0.3f) * 1.01f + 0.33f) * 1.01f + 2.0f;
    const float u = j00 * tx + c.cx, v = j11 * ty + c.cy;
    return u + rb < 0.0f || u - rb > (float)(W - 1) || v + rb < 0.0f || v - rb > (float)(H - 1);
}

// Largest absolute scale of Gaussian g (FP32 or FP16 storage): the only attribute the
// off-screen test reads besides the mean.
__device__ __forceinline__ float load_max_scale(const cgs_scene& S, long long g)
{
    float s0, s1, s2;
    if (S.attr_fp16) {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(S.scale) + g);
        s0 = h2f(a.x & 0xffffu);
        s1 = h2f(a.x >> 16);
        s2 = h2f(a.y & 0xffffu);
    } else {
        const float4 a = __ldg(reinterpret_cast<const float4*>(S.scale) + g);
        s0 = a.x;
        s1 = a.y;
        s2 = a.z;
    }
    return fmaxf(fmaxf(fabsf(s0), fabsf(s1)), fabsf(s2));
}

// L2 prefetch of the rows phase 2 reads for a candidate: its SH coefficients (one 192-byte
// row at degree 3 in FP32, which spans two 128-byte lines) and its rotation.
template <int DEG>
__device__ __forceinline__ void prefetch_rows(const cgs_scene& S, long long g)
{
    constexpr int nc = (DEG + 1) * (DEG + 1);
    const size_t row = (size_t)(nc * 3) * (S.attr_fp16 ? 2u : 4u);
    const char* p = reinterpret_cast<const char*>(S.sh) + (size_t)g * row;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    if (row > 64) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + row - 1));
    const char* q = reinterpret_cast<const char*>(S.quat) + (size_t)g * (S.attr_fp16 ? 8u : 16u);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
}

// The CTA walks the selected list (flattened over views) in steps of PROJ_STEP Gaussians (a
// uniform trip count, so the CTA-wide steps below are safe).
//   phase 1  PROJ_ITEMS Gaussians per thread: scene index, near plane, the point-wise level
//            test, the cheap off-screen bound; the survivors are queued in shared memory
//   phase 2  in rounds of one queued Gaussian per thread (dense warps, so the full projection
//            is not run by warps whose lanes are mostly culled; survivors of several steps are
//            queued until a full round is there, so a step whose few survivors would fill a
//            fraction of a round runs no phase 2 at all): covariance,
//            radius, tile rect; for the visible ones the projected record (screen-space part
//            and the view-dependent SH colour, Sec. 3.1, its coefficients read as they are
//            used), the rect and the (view, depth) sort key
//   phase 3  compaction and duplication: the CTA sums its visible count and tiles touched
//            (warp ballots and shuffles, then the warp totals in shared memory) and reserves a
//            range of the visible list and of the entry buffer with one atomic add each; the
//            whole CTA then emits the round's (tile << 32 | j) entries: thread t takes entries
//            t, t + 128, ..., finds the owning Gaussian by a binary search over the round's
//            exclusive offsets in shared memory, and counts the tile (in the sub-range of the
//            entry's index).  A round of large
//            Gaussians (hundreds of tiles each, near the camera) is spread over all warps.
// The order of the visible list and of the entries depends on the order in which CTAs
// reserve their ranges; nothing downstream depends on it (entries are sorted per tile by
// (depth, index), the backward works per Gaussian).  DEG is the scene's SH degree.
constexpr int PROJ_THREADS = 128;
constexpr int PROJ_WARPS = PROJ_THREADS / 32;
constexpr int PROJ_ITEMS = 2;  // selected Gaussians per thread in phase 1
constexpr int PROJ_STEP = PROJ_THREADS * PROJ_ITEMS;
constexpr int PROJ_CTAS_PER_SM = 10;  // latency-bound: registers capped so ten CTAs fit an SM

template <int DEG>
__global__ void __launch_bounds__(PROJ_THREADS, PROJ_CTAS_PER_SM)
    k_project(Layout L, cgs_scene S, const cgs_camera* __restrict__ cams, float near_z)
{
    __shared__ uint32_t s_wv[PROJ_WARPS], s_wt[PROJ_WARPS];
    __shared__ uint32_t s_vbase, s_nq, s_rtot;
    __shared__ uint32_t s_ex[PROJ_THREADS], s_ej[PROJ_THREADS], s_rx[PROJ_THREADS], s_ry[PROJ_THREADS];
    __shared__ int s_ev[PROJ_THREADS];
    __shared__ unsigned long long s_ebase;
    // the queue of phase-1 survivors: a remainder of fewer than PROJ_THREADS from earlier steps
    // plus one step's survivors
    constexpr int QCAP = PROJ_STEP + PROJ_THREADS;
    __shared__ uint32_t s_qj[QCAP];
    __shared__ int s_qv[QCAP];
    __shared__ long long s_qg[QCAP];
    const uint32_t n = L.hdr->n_sel;
    const float4* __restrict__ mo4 = reinterpret_cast<const float4*>(S.mean_opac);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const unsigned long long cap = (unsigned long long)L.k_cap;
    if (threadIdx.x == 0) s_nq = 0;
    __syncthreads();
    for (uint32_t base = blockIdx.x * PROJ_STEP; base < n; base += gridDim.x * PROJ_STEP) {
        const bool last_step = base + gridDim.x * PROJ_STEP >= n;  // this CTA's final step (uniform)
        // phase 1: survivors appended to the queue
#pragma unroll 1
        for (int u = 0; u < PROJ_ITEMS; u++) {
            const uint32_t j = base + (uint32_t)(u * PROJ_THREADS) + threadIdx.x;
            bool cand = false;
            int v = 0;
            long long g = 0;
            if (j < n) {
                locate(L, j, &v, &g);
                L.gidx[j] = (uint32_t)g;
                const cgs_camera& c = cams[v];
                // the scale row is read with the position, not after the near-plane test: one
                // round trip instead of two for the Gaussians in front of the camera
                const float4 mo = __ldg(mo4 + g);
                const float sm0 = load_max_scale(S, g);
                const float m[3] = {mo.x, mo.y, mo.z};
                const float tz = ((c.R[6] * m[0] + c.R[7] * m[1]) + c.R[8] * m[2]) + c.t[2];
                bool keep = tz > near_z;
                if (keep && L.lod_mode == CGS_LOD_POINT) {
                    // point-wise baseline: the level of this Gaussian's own distance; kept iff
                    // its rank in the block lies inside that level's (nested) prefix
                    const float d0 = m[0] - c.campos[0], d1 = m[1] - c.campos[1], d2 = m[2] - c.campos[2];
                    const float dist = sqrtf((d0 * d0 + d1 * d1) + d2 * d2);
                    int lv = dist < L.lod_d1 ? 0 : (dist < L.lod_d2 ? 1 : 2);
                    if (lv > S.n_levels - 1) lv = S.n_levels - 1;
                    int blk;
                    uint32_t rank;
                    locate_block(L, j, v, &blk, &rank);
                    keep = (long long)rank < S.level_count[(long long)blk * S.n_levels + lv];
                }
                if (keep) {
                    const float sm = sm0;
                    const float tx = ((c.R[0] * m[0] + c.R[1] * m[1]) + c.R[2] * m[2]) + c.t[0];
                    const float ty = ((c.R[3] * m[0] + c.R[4] * m[1]) + c.R[5] * m[2]) + c.t[1];
                    keep = !surely_off_screen(sm, c, tx, ty, tz, L.W, L.H);
                }
                cand = keep;
                if (!cand) L.tt[j] = 0;
            }
            const uint32_t cb = __ballot_sync(0xffffffffu, cand);
            uint32_t wbase = 0;
            if (lane == 0 && cb) wbase = atomicAdd(&s_nq, (uint32_t)__popc(cb));
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            if (cand) {
                const uint32_t slot = wbase + __popc(cb & lt);
                s_qj[slot] = j;
                s_qv[slot] = v;
                s_qg[slot] = g;
                // the rows of phase 2's first round, fetched into L2 while phase 1 goes on
                if (slot < PROJ_THREADS) prefetch_rows<DEG>(S, g);
            }
        }
        __syncthreads();
        const uint32_t nq = s_nq;
        // phase 2 runs full rounds only; the rest waits in the queue for the next step's
        // survivors (all of it in the CTA's last step)
        const uint32_t nproc = last_step ? nq : (nq / PROJ_THREADS) * PROJ_THREADS;
        __syncthreads();  // every thread has read nq before the queue is compacted below
        for (uint32_t q0 = 0; q0 < nproc; q0 += PROJ_THREADS) {
            // phase 2
            uint32_t tt = 0, rx = 0, ry = 0, j = 0;
            int v = 0;
            if (q0 + threadIdx.x < nproc) {
                const uint32_t qi = q0 + threadIdx.x;
                j = s_qj[qi];
                v = s_qv[qi];
                const long long g = s_qg[qi];
                const cgs_camera& c = cams[v];
                const float4 mo = __ldg(mo4 + g);
                const float m[3] = {mo.x, mo.y, mo.z};
                float s[3], q[4];
                load_scale_quat(S, g, s, q);
                Proj p;
                if (project_one(m, s, q, c, near_z, p) == 0) {
                    const float r = ceilf(3.0f * sqrtf(p.lam1));
                    const float W1 = (float)(L.W - 1), H1 = (float)(L.H - 1);
                    float x0 = ceilf(p.u - r), x1 = floorf(p.u + r);
                    float y0 = ceilf(p.v - r), y1 = floorf(p.v + r);
                    if (x0 < 0.0f) x0 = 0.0f;
                    if (y0 < 0.0f) y0 = 0.0f;
                    if (x1 > W1) x1 = W1;
                    if (y1 > H1) y1 = H1;
                    if (x0 <= x1 && y0 <= y1) {
                        const uint32_t tx0 = (uint32_t)x0 / L.B, tx1 = (uint32_t)x1 / L.B + 1;
                        const uint32_t ty0 = (uint32_t)y0 / L.B, ty1 = (uint32_t)y1 / L.B + 1;
                        tt = (tx1 - tx0) * (ty1 - ty0);
                        rx = tx0 | (ty0 << 16);
                        ry = tx1 | (ty1 << 16);
                        L.rect[j] = make_uint2(rx, ry);
                        float ex, ey, tq;
                        cull_extent(mo.w, p.A, p.B, p.C, &ex, &ey, &tq);
                        L.rec[3 * (size_t)j] = make_float4(p.u, p.v, mo.w, ex);
                        L.rec[3 * (size_t)j + 1] = make_float4(p.conic[0], p.conic[1], p.conic[2], ey);
                        float rgb[3];
                        sh_colour_streamed<DEG>(m, c, S, g, rgb);
                        L.rec[3 * (size_t)j + 2] = make_float4(rgb[0], rgb[1], rgb[2], tq);
                        L.pkey[j] = ((unsigned long long)(uint32_t)v << 32) | __float_as_uint(p.tz);
                    }
                }
                L.tt[j] = tt;
            }
            // phase 3: warp totals, visible count (ballot) and tiles touched (inclusive shuffle scan)
            const uint32_t vb = __ballot_sync(0xffffffffu, tt > 0);
            uint32_t inc = tt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint32_t excl = inc - tt;
            const uint32_t wtot = __shfl_sync(0xffffffffu, inc, 31);
            if (lane == 0) {
                s_wv[warp] = __popc(vb);
                s_wt[warp] = wtot;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t nv = 0;
                unsigned long long ne = 0;
                for (int w = 0; w < PROJ_WARPS; w++) {
                    const uint32_t a = s_wv[w], b = s_wt[w];
                    s_wv[w] = nv;
                    s_wt[w] = (uint32_t)ne;
                    nv += a;
                    ne += b;
                }
                s_vbase = nv ? atomicAdd(&L.hdr->n_vis, nv) : 0u;
                s_ebase = ne ? atomicAdd(&L.hdr->k_total, ne) : 0ull;
                s_rtot = (uint32_t)ne;
                if (ne && s_ebase + ne > cap) latch(L.hdr, ST_CAPACITY);
            }
            __syncthreads();
            if (tt > 0) L.vis[s_vbase + s_wv[warp] + __popc(vb & lt)] = j;
            // the round's entries, emitted by the whole CTA: each thread's Gaussian in shared
            // memory with its exclusive entry offset in the round
            s_ex[threadIdx.x] = s_wt[warp] + excl;
            s_ej[threadIdx.x] = j;
            s_ev[threadIdx.x] = v;
            s_rx[threadIdx.x] = rx;
            s_ry[threadIdx.x] = ry;
            __syncthreads();
            const uint32_t rtot = s_rtot;
            for (uint32_t idx = threadIdx.x; idx < rtot; idx += PROJ_THREADS) {
                // owner: the last slot o with s_ex[o] <= idx (a slot with no entries shares its
                // successor's offset and is never the last such slot)
                int o = 0;
#pragma unroll
                for (int step = PROJ_THREADS / 2; step >= 1; step >>= 1)
                    if (s_ex[o + step] <= idx) o += step;
                const unsigned long long k = s_ebase + idx;
                if (k < cap) {
                    const uint32_t orx = s_rx[o], ory = s_ry[o];
                    const uint32_t tx0 = orx & 0xffffu, ty0 = orx >> 16, w = (ory & 0xffffu) - tx0;
                    const uint32_t local = idx - s_ex[o];
                    const uint32_t t = (uint32_t)s_ev[o] * (uint32_t)L.T + (ty0 + local / w) * (uint32_t)L.tiles_x +
                                       (tx0 + local % w);
                    L.eraw[k] = ((unsigned long long)t << 32) | s_ej[o];
                    atomicAdd(&L.tcnt[((size_t)t << L.tsub_sh) + (s_ej[o] & ((1u << L.tsub_sh) - 1u))], 1u);
                }
            }
            __syncthreads();
        }
        // the unprocessed remainder (fewer than PROJ_THREADS) moves to the front of the queue;
        // its rows are fetched into L2 for the next step's first round
        if (nproc > 0 && nproc < nq) {
            const uint32_t rem = nq - nproc;
            uint32_t qj = 0;
            int qv = 0;
            long long qg = 0;
            if (threadIdx.x < rem) {
                qj = s_qj[nproc + threadIdx.x];
                qv = s_qv[nproc + threadIdx.x];
                qg = s_qg[nproc + threadIdx.x];
            }
            __syncthreads();
            if (threadIdx.x < rem) {
                s_qj[threadIdx.x] = qj;
                s_qv[threadIdx.x] = qv;
                s_qg[threadIdx.x] = qg;
                prefetch_rows<DEG>(S, qg);
            }
        }
        if (threadIdx.x == 0) s_nq = nq - nproc;
        __syncthreads();
    }
}

void launch_project(const Layout& L, const cgs_scene& S, const cgs_camera* cams, float near_z, int n_sm,
                    cudaStream_t st)
{
    long long want = (L.n_cap + PROJ_STEP - 1) / PROJ_STEP;
    long long grid = want < (long long)n_sm * PROJ_CTAS_PER_SM ? want : (long long)n_sm * PROJ_CTAS_PER_SM;
    if (grid < 1) grid = 1;
    switch (S.sh_degree) {
        case 0: k_project<0><<<(unsigned)grid, PROJ_THREADS, 0, st>>>(L, S, cams, near_z); break;
        case 1: k_project<1><<<(unsigned)grid, PROJ_THREADS, 0, st>>>(L, S, cams, near_z); break;
        case 2: k_project<2><<<(unsigned)grid, PROJ_THREADS, 0, st>>>(L, S, cams, near_z); break;
        default: k_project<3><<<(unsigned)grid, PROJ_THREADS, 0, st>>>(L, S, cams, near_z); break;
    }
}



}  // namespace cgs
