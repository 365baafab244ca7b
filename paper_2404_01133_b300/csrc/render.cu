// Stage d of the hot path: per-tile front-to-back alpha compositing (Eq. 1, Sec. 3.1), plus
// the L1 loss (Sec. 3.2.3).  The CTA leaves as soon as every pixel stopped
// (__syncthreads_count).
#include "render_common.cuh"

namespace cgs {

// Forward.  Staging a batch, each loading thread also records which warps its Gaussian can
// reach; each warp then visits only those entries (ballot over 32-entry chunks), in list
// order.  n_contrib and the evaluated-pair count keep the semantics of a walk over the full
// list: entries up to and including the stopping one, or the whole list.
//
// A lane's two pixels are packed pairs (render_common.cuh): the falloff, -alpha, the
// transmittance update and the colour sums of both pixels take one packed instruction each.
// The colour is accumulated negated (the staged opacity is -o), NC = -C, exactly.  Per pixel
// and entry, written without branches: a warp runs every step for all its lanes anyway, and
// a pair that does not blend adds c * 0 and keeps T and last.
//
// With HITS, every blend is also counted per scene Gaussian: one atomic add per (warp, entry)
// of the number of the warp's pixels that blended it (L.hits, indexed by scene index).
template <int B, int BATCH, bool HITS, bool EXACT>
__global__ void __launch_bounds__(B * B / 2, B == 16 ? 8 : 32) k_render_fwd(Layout L, const uint32_t* __restrict__ tval, float bg0,
                                                          float bg1, float bg2, float* __restrict__ image,
                                                          float* __restrict__ final_T, uint32_t* __restrict__ n_contrib)
{
    constexpr int NT = B * B / 2;
    __shared__ float4 s_e0[BATCH], s_e1[BATCH], s_e2[BATCH], s_e3[BATCH];
    __shared__ uint32_t s_m[BATCH];
    __shared__ uint32_t s_g[HITS ? BATCH : 1];
    __shared__ float4 s_cn[EXACT ? BATCH : 1];  // parity build: conic A', B', C' and opacity
    const int v = blockIdx.z;
    const int tile = blockIdx.y * L.tiles_x + blockIdx.x;
    const uint2 rg = reinterpret_cast<const uint2*>(L.ranges)[(size_t)v * L.T + tile];
    int lx, ly, wx0, wy0;
    pixels_of<B>(threadIdx.x, &lx, &ly, &wx0, &wy0);
    const int px = blockIdx.x * B + lx, py0 = blockIdx.y * B + ly, py1 = py0 + 4;
    const bool in0 = px < L.W && py0 < L.H, in1 = px < L.W && py1 < L.H;
    const float fpx = (float)px;
    const float2 fpy = make_float2((float)py0, (float)py1);
    const float tx0 = (float)(blockIdx.x * B), ty0 = (float)(blockIdx.y * B);
    const int lane = threadIdx.x & 31;
    const uint32_t wbit = 1u << (threadIdx.x >> 5);
    // this warp's contribution words: NW * (start / 32 + tile index) + warp * (len / 32 + 1)
    constexpr int NW = B * B / 64;
    const size_t tg = (size_t)v * L.T + tile;
    uint32_t* cbits = L.cbits + (size_t)NW * (rg.x / 32 + tg) + (size_t)(threadIdx.x >> 5) * ((rg.y - rg.x) / 32 + 1);
    uint32_t steps = 0, useful = 0;  // warp steps visited / with a blend (lane 0 counts)
    float2 T = make_float2(1.0f, 1.0f);
    float2 NC0 = make_float2(0.0f, 0.0f), NC1 = NC0, NC2 = NC0;  // minus the colour sums
    uint32_t last0 = 0, last1 = 0, stop0 = 0xffffffffu, stop1 = 0xffffffffu;
    bool done0 = !in0, done1 = !in1;
    const float nthr = -1.0f / 255.0f;
    for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
        if (__syncthreads_count(done0 && done1) == NT) break;
        for (int i = threadIdx.x; i < BATCH; i += NT) {
            uint32_t m = 0;
            if (start + i < rg.y) {
                const size_t j = tval[start + i];
                const float4 a = L.rec[3 * j], b = L.rec[3 * j + 1], c = L.rec[3 * j + 2];
                const Staged se = stage_entry(a, b, c);
                s_e0[i] = se.e0;
                s_e1[i] = se.e1;
                s_e2[i] = se.e2;
                s_e3[i] = se.e3;
                m = warp_mask<B>(a, b, c.w, tx0, ty0);
                if (HITS) s_g[i] = L.gidx[j];
                if (EXACT) s_cn[i] = make_float4(b.x, b.y, b.z, a.z);
            }
            s_m[i] = m;
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)BATCH, rg.y - start);
        for (int c0 = 0; c0 < nb; c0 += 32) {
            if (__all_sync(0xffffffffu, done0 && done1)) break;
            uint32_t bits = __ballot_sync(0xffffffffu, c0 + lane < nb && (s_m[c0 + lane] & wbit));
            const uint32_t s_bits = bits;
            uint32_t word = 0;
            while (bits) {
                const int kk = __ffs(bits) - 1;
                bits &= bits - 1;
                const int k = c0 + kk;
                const float4 e0 = s_e0[k], e1 = s_e1[k], e2 = s_e2[k], e3 = s_e3[k];
                const uint32_t pos = start - rg.x + (uint32_t)k;
                float2 p, na, Tn;  // power (times log2 e in the fast path), -alpha, T (1 - alpha)
                if constexpr (EXACT) {
                    const float4 cn = s_cn[k];
                    p = make_float2(exact_power(cn, e1.x, e0.x, fpx, fpy.x), exact_power(cn, e1.x, e0.x, fpx, fpy.y));
                    const float a0 = exact_alpha(exact_og(cn.w, p.x)), a1 = exact_alpha(exact_og(cn.w, p.y));
                    na = make_float2(-a0, -a1);
                    Tn = make_float2(ieee_mul(T.x, ieee_sub(1.0f, a0)), ieee_mul(T.y, ieee_sub(1.0f, a1)));
                } else {
                    float dx;
                    float2 dy;
                    p = staged_power2(e0, e1, fpx, fpy, &dx, &dy);
                    const float2 G = make_float2(gauss_exp2(p.x), gauss_exp2(p.y));
                    float2 nog;
                    na = neg_alpha2(e2, G, &nog);  // -alpha
                    Tn = ieee_fma2(na, T, T);      // T (1 - alpha), rounded once
                }
                const bool ok0 = !done0 && !(p.x > 0.0f) && !(na.x > nthr);
                const bool ok1 = !done1 && !(p.y > 0.0f) && !(na.y > nthr);
                const bool st0 = ok0 && Tn.x < 1e-4f, st1 = ok1 && Tn.y < 1e-4f;
                const bool b0 = ok0 && !st0, b1 = ok1 && !st1;
                if constexpr (EXACT) {
                    // the colour sums C + c (alpha T), positive in this build
                    if (b0) {
                        const float w = ieee_mul(-na.x, T.x);
                        NC0.x = ieee_add(NC0.x, ieee_mul(e2.z, w));
                        NC1.x = ieee_add(NC1.x, ieee_mul(e3.x, w));
                        NC2.x = ieee_add(NC2.x, ieee_mul(e3.z, w));
                        T.x = Tn.x;
                    }
                    if (b1) {
                        const float w = ieee_mul(-na.y, T.y);
                        NC0.y = ieee_add(NC0.y, ieee_mul(e2.w, w));
                        NC1.y = ieee_add(NC1.y, ieee_mul(e3.y, w));
                        NC2.y = ieee_add(NC2.y, ieee_mul(e3.w, w));
                        T.y = Tn.y;
                    }
                } else {
                    // -alpha where the pixel blends, 0 where it does not: then T (1 - alpha) and the
                    // colour weight alpha T come out of the packed FMA pipe (fma(0, T, T) = T exactly)
                    const float2 nab = make_float2(b0 ? na.x : 0.0f, b1 ? na.y : 0.0f);
                    const float2 w = __fmul2_rn(nab, T);        // -alpha T, or 0
                    NC0 = __ffma2_rn(make_float2(e2.z, e2.w), w, NC0);
                    NC1 = __ffma2_rn(make_float2(e3.x, e3.y), w, NC1);
                    NC2 = __ffma2_rn(make_float2(e3.z, e3.w), w, NC2);
                    T = ieee_fma2(nab, T, T);
                }
                last0 = b0 ? pos + 1u : last0;
                last1 = b1 ? pos + 1u : last1;
                stop0 = st0 ? pos : stop0;
                stop1 = st1 ? pos : stop1;
                done0 = done0 || st0;
                done1 = done1 || st1;
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
    if constexpr (EXACT) {
        // C + T bg as the plain loop forms it; stored negated to share the writes below
        NC0 = make_float2(-ieee_add(NC0.x, ieee_mul(T.x, bg0)), -ieee_add(NC0.y, ieee_mul(T.y, bg0)));
        NC1 = make_float2(-ieee_add(NC1.x, ieee_mul(T.x, bg1)), -ieee_add(NC1.y, ieee_mul(T.y, bg1)));
        NC2 = make_float2(-ieee_add(NC2.x, ieee_mul(T.x, bg2)), -ieee_add(NC2.y, ieee_mul(T.y, bg2)));
        bg0 = bg1 = bg2 = 0.0f;
    }
    if (in0) {
        const size_t pix = (size_t)py0 * L.W + px;
        image[(3 * (size_t)v + 0) * HW + pix] = T.x * bg0 - NC0.x;
        image[(3 * (size_t)v + 1) * HW + pix] = T.x * bg1 - NC1.x;
        image[(3 * (size_t)v + 2) * HW + pix] = T.x * bg2 - NC2.x;
        final_T[(size_t)v * HW + pix] = T.x;
        n_contrib[(size_t)v * HW + pix] = last0;
    }
    if (in1) {
        const size_t pix = (size_t)py1 * L.W + px;
        image[(3 * (size_t)v + 0) * HW + pix] = T.y * bg0 - NC0.y;
        image[(3 * (size_t)v + 1) * HW + pix] = T.y * bg1 - NC1.y;
        image[(3 * (size_t)v + 2) * HW + pix] = T.y * bg2 - NC2.y;
        final_T[(size_t)v * HW + pix] = T.y;
        n_contrib[(size_t)v * HW + pix] = last1;
    }
    const uint32_t len = rg.y - rg.x;
    const uint32_t visited = (in0 ? (stop0 != 0xffffffffu ? stop0 + 1u : len) : 0u) +
                             (in1 ? (stop1 != 0xffffffffu ? stop1 + 1u : len) : 0u);
    const uint32_t ws = __reduce_add_sync(0xffffffffu, visited);
    if (lane == 0) {
        if (ws) atomicAdd(&L.hdr->pairs_fwd, (unsigned long long)ws);
        if (steps) atomicAdd(&L.hdr->steps_fwd, (unsigned long long)steps);
        if (useful) atomicAdd(&L.hdr->steps_useful, (unsigned long long)useful);
    }
}

template <int B, int BATCH>
static void fwd_launch(const Layout& L, const uint32_t* tval, const cgs_config& c, float* img, float* T, uint32_t* nc,
                       cudaStream_t st)
{
    dim3 grid(L.tiles_x, L.tiles_y, L.V);
    if (c.exact)
        k_render_fwd<B, BATCH, false, true><<<grid, B * B / 2, 0, st>>>(L, tval, c.bg[0], c.bg[1], c.bg[2], img, T, nc);
    else if (L.hits)
        k_render_fwd<B, BATCH, true, false><<<grid, B * B / 2, 0, st>>>(L, tval, c.bg[0], c.bg[1], c.bg[2], img, T, nc);
    else
        k_render_fwd<B, BATCH, false, false><<<grid, B * B / 2, 0, st>>>(L, tval, c.bg[0], c.bg[1], c.bg[2], img, T, nc);
}
bool launch_render_fwd(const Layout& L, const cgs_config& c, float* img, float* T, uint32_t* nc, cudaStream_t st)
{
    const uint32_t* tv = L.tval;
    if (c.exact && L.hits) return false;  // hit counting has no parity build
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

// The falloff exponential of both compositing kernels (gauss_exp2) over an array, for the
// tests that bound its error.
__global__ void __launch_bounds__(256) k_debug_exp2(const float* __restrict__ p, long long n, float* __restrict__ g)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        g[i] = gauss_exp2(p[i]);
}

void launch_debug_exp2(const float* p, long long n, float* g, int n_sm, cudaStream_t st)
{
    long long grid = (n + 255) / 256;
    if (grid > (long long)n_sm * 16) grid = (long long)n_sm * 16;
    if (grid < 1) grid = 1;
    k_debug_exp2<<<(unsigned)grid, 256, 0, st>>>(p, n, g);
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
