// Backward of stage d (differentiable rendering, Sec. 3.1): every pixel replays its blended
// entries back to front from its final transmittance and n_contrib.  Built with
// flush-to-zero (denormal results of the gradient arithmetic become zero; the decisions that
// must match the forward are computed by render_common.cuh's explicit IEEE instructions or
// do not depend on denormals: a denormal exp() or opacity product is below 1/255 either way).
#include "render_common.cuh"

namespace cgs {

// A target value of the fused L1 loss, as stored: FP32 (LOSS = 2), or the 8-bit channel value
// (LOSS = 1) mapped through the shared t / 255 table later.
template <int LOSS>
__device__ __forceinline__ float l1_target(const void* tgt, size_t i)
{
    if constexpr (LOSS == 1) return (float)static_cast<const uint8_t*>(tgt)[i];
    else return static_cast<const float*>(tgt)[i];
}

// *g holds the image value on entry and the L1 gradient sign(img - target) inv on return
// (0 where they are equal or either is NaN); returns |img - target|.  Explicit IEEE subtract
// and non-flushing compares, as in cgs_l1_loss.
template <int LOSS>
__device__ __forceinline__ float l1_grad(float* g, float t, const float* tab, float inv)
{
    const float tv = LOSS == 1 ? tab[(int)t] : t;
    const float d = ieee_sub(*g, tv);
    float r;
    asm("{\n\t.reg .pred gt, lt;\n\t"
        "setp.gt.f32 gt, %1, 0f00000000;\n\t"
        "setp.lt.f32 lt, %1, 0f00000000;\n\t"
        "selp.f32 %0, %2, 0f00000000, gt;\n\t"
        "@lt mov.f32 %0, %3;\n\t}"
        : "=f"(r)
        : "f"(d), "f"(inv), "f"(-inv));
    *g = r;
    return fabsf(d);
}

// Backward.  A warp visits exactly the entries that blended into at least one of its pixels
// in the forward (the forward's contribution bits), last first.  Per entry, a lane replays its
// two pixels as packed pairs and reduces them to nine values:
//   w = dL/do of a pixel (dalpha/do = G when the 0.99 clamp is inactive, else 0); since
//   dL/dpower = o w, the power moments are kept as moments of w:  m0 = sum w dx,
//   m1 = sum w dy, m2 = sum w dx^2, m3 = sum w dx dy, m4 = sum w dy^2, m5 = sum w;
//   m6..m8 = sum (-alpha T) dL/d(r, g, b)  (negated colour gradient, the staged opacity
//   being -o).
// The two pixels of a lane share dx, so m0 = dx m5, m2 = dx m0, m3 = dx m1.  Up to three
// entries' 27 values go through a per-warp shared-memory transpose (row = value, column =
// lane; lane r then sums row r with eight 16-byte loads), and lane 9 e + c adds the warp's sum
// of m_c for entry e to the Gaussian's row of the global accumulator (one vector of 27 atomic
// adds per three entries).  The moments are linear in the pixels, so the projection backward
// turns their totals into dL/d(u, v, conic, o, rgb) once per Gaussian, with its conic and
// opacity: no per-tile flush, no shared accumulator, no barrier after the replay.
//
// Replay of one pixel: from its final transmittance T and gS = dL/dP . S, S the colour behind
// the current entry (initially T_final bg), entry i with alpha = min(0.99, o G) recovers
// T_before = T / (1 - alpha); dL/dalpha = (T (g . c) - gS) / (1 - alpha), dL/dc = g alpha
// T_before; then T = T_before and gS += alpha T_before (g . c).  The running sum is kept
// negated (ngS = -gS) and alpha enters as -alpha, so no step negates anything.
//
// LOSS = 0: dL/dimage is read from dL_dimg.  LOSS = 1 (8-bit target) or 2 (FP32 target): it is
// the L1 gradient sign(img - target) / count (L1In), formed here from l1.img and l1.tgt, and the
// CTA's share of mean |img - target| goes to *l1.loss; dL_dimg is not read.  The difference and
// both sign tests are explicit IEEE instructions, so this file's flush-to-zero leaves the
// gradient bit-identical to cgs_l1_loss's.
//
// COUNT: the contributing pairs replayed are counted into the frame header (a diagnostic).
template <int B, int BATCH, bool EXACT, int LOSS, bool COUNT>
__global__ void __launch_bounds__(B * B / 2, B == 16 ? 7 : 28) k_render_bwd(Layout L, const uint32_t* __restrict__ tval, float bg0,
                                                          float bg1, float bg2, const float* __restrict__ dL_dimg,
                                                          const float* __restrict__ final_T,
                                                          const uint32_t* __restrict__ n_contrib, L1In l1)
{
    constexpr int NT = B * B / 2;
    constexpr int NW = B * B / 64;
    constexpr int RS = 36;  // transpose row stride: 32 lanes + 4, conflict-free 16-byte row reads
    __shared__ float4 s_e0[BATCH], s_e1[BATCH], s_e2[BATCH], s_e3[BATCH];
    __shared__ float4 s_cn[EXACT ? BATCH : 1];  // parity build: conic A', B', C' and opacity
    __shared__ uint32_t s_j[BATCH];
    __shared__ uint8_t s_pos[NW][BATCH];  // per warp: the batch positions it visits, highest first
    __shared__ __align__(16) float s_red[NW][27][RS];
    __shared__ uint32_t s_maxnc;
    __shared__ float s_tab[LOSS == 1 ? 256 : 1];  // t / 255 for an 8-bit target, correctly rounded
    __shared__ float s_lw[LOSS ? NW : 1];         // per-warp sums of |img - target|
    const int v = blockIdx.z;
    const int tile = blockIdx.y * L.tiles_x + blockIdx.x;
    const uint2 rg = reinterpret_cast<const uint2*>(L.ranges)[(size_t)v * L.T + tile];
    int lx, ly, wx0, wy0;
    pixels_of<B>(threadIdx.x, &lx, &ly, &wx0, &wy0);
    const int px = blockIdx.x * B + lx, py0 = blockIdx.y * B + ly, py1 = py0 + 4;
    const bool in0 = px < L.W && py0 < L.H, in1 = px < L.W && py1 < L.H;
    const float fpx = (float)px;
    const float2 fpy = make_float2((float)py0, (float)py1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t tg = (size_t)v * L.T + tile;
    const uint32_t* cbits = L.cbits + (size_t)NW * (rg.x / 32 + tg) + (size_t)warp * ((rg.y - rg.x) / 32 + 1);
    const size_t HW = (size_t)L.W * L.H;
    float2 T = make_float2(1.0f, 1.0f), g0 = make_float2(0.0f, 0.0f), g1 = g0, g2 = g0;
    uint32_t nc0 = 0, nc1 = 0;
    // with LOSS: the image values in g*, the target values (raw) in t*, turned into the
    // gradient after the first barrier (the 8-bit table is built before it)
    float2 t0 = g0, t1 = g0, t2 = g0;
    if (in0) {
        const size_t pix = (size_t)py0 * L.W + px;
        T.x = final_T[(size_t)v * HW + pix];
        nc0 = n_contrib[(size_t)v * HW + pix];
        const float* src = LOSS ? l1.img : dL_dimg;
        g0.x = src[(3 * (size_t)v + 0) * HW + pix];
        g1.x = src[(3 * (size_t)v + 1) * HW + pix];
        g2.x = src[(3 * (size_t)v + 2) * HW + pix];
        if constexpr (LOSS) {
            t0.x = l1_target<LOSS>(l1.tgt, (3 * (size_t)v + 0) * HW + pix);
            t1.x = l1_target<LOSS>(l1.tgt, (3 * (size_t)v + 1) * HW + pix);
            t2.x = l1_target<LOSS>(l1.tgt, (3 * (size_t)v + 2) * HW + pix);
        }
    }
    if (in1) {
        const size_t pix = (size_t)py1 * L.W + px;
        T.y = final_T[(size_t)v * HW + pix];
        nc1 = n_contrib[(size_t)v * HW + pix];
        const float* src = LOSS ? l1.img : dL_dimg;
        g0.y = src[(3 * (size_t)v + 0) * HW + pix];
        g1.y = src[(3 * (size_t)v + 1) * HW + pix];
        g2.y = src[(3 * (size_t)v + 2) * HW + pix];
        if constexpr (LOSS) {
            t0.y = l1_target<LOSS>(l1.tgt, (3 * (size_t)v + 0) * HW + pix);
            t1.y = l1_target<LOSS>(l1.tgt, (3 * (size_t)v + 1) * HW + pix);
            t2.y = l1_target<LOSS>(l1.tgt, (3 * (size_t)v + 2) * HW + pix);
        }
    }
    if (threadIdx.x == 0) s_maxnc = 0;
    if constexpr (LOSS == 1)
        for (int i = threadIdx.x; i < 256; i += NT) s_tab[i] = __fdiv_rn((float)i, 255.0f);
    __syncthreads();
    if constexpr (LOSS) {
        float acc = 0.0f;
        if (in0) {
            acc += l1_grad<LOSS>(&g0.x, t0.x, s_tab, l1.inv);
            acc += l1_grad<LOSS>(&g1.x, t1.x, s_tab, l1.inv);
            acc += l1_grad<LOSS>(&g2.x, t2.x, s_tab, l1.inv);
        }
        if (in1) {
            acc += l1_grad<LOSS>(&g0.y, t0.y, s_tab, l1.inv);
            acc += l1_grad<LOSS>(&g1.y, t1.y, s_tab, l1.inv);
            acc += l1_grad<LOSS>(&g2.y, t2.y, s_tab, l1.inv);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_lw[warp] = acc;
    }
    float2 ngS = make_float2(-(T.x * (g0.x * bg0 + g1.x * bg1 + g2.x * bg2)),
                             -(T.y * (g0.y * bg0 + g1.y * bg1 + g2.y * bg2)));
    const uint32_t mnc = max(nc0, nc1);
    if (mnc) atomicMax(&s_maxnc, mnc);
    __syncthreads();
    if constexpr (LOSS) {
        if (threadIdx.x == 0) {
            float t = 0.0f;
#pragma unroll
            for (int w = 0; w < NW; w++) t += s_lw[w];
            if (t != 0.0f) atomicAdd(l1.loss, t * l1.inv);
        }
    }
    const long long first = rg.x;
    // n_contrib never exceeds the tile's list length; clamp so a mismatched buffer cannot
    // move the replay outside this tile's entries
    const long long end = (first + s_maxnc) < (long long)rg.y ? (first + s_maxnc) : (long long)rg.y;
    // the forward wrote this warp's contribution words up to its last blended position
    uint32_t wmax = mnc;
#pragma unroll
    for (int o = 16; o; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    const float nthr = -1.0f / 255.0f;
    const float2 one = make_float2(1.0f, 1.0f);
    uint32_t pairs = 0;
    float(*red)[RS] = s_red[warp];
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
            const float4 a = L.rec[3 * (size_t)j], cb = L.rec[3 * (size_t)j + 1], c = L.rec[3 * (size_t)j + 2];
            const Staged se = stage_entry(a, cb, c);
            s_e0[i] = se.e0;
            s_e1[i] = se.e1;
            s_e2[i] = se.e2;
            s_e3[i] = se.e3;
            if (EXACT) s_cn[i] = make_float4(cb.x, cb.y, cb.z, a.z);
        }
        __syncthreads();
        const int kmax = (int)min((long long)nb, (long long)wmax - (bs - first));  // entries k < kmax
        // this warp's set bits of the batch as a list of positions, highest first: lane c holds
        // the contribution word of the batch's chunk c, and each chunk's set bits (taken highest
        // first, one per lane) are placed by a ballot
        uint8_t* pos = s_pos[warp];
        int cnt = 0;
        if (kmax > 0) {
            const int nwords = (kmax + 31) >> 5;
            uint32_t word = 0;
            if (lane < nwords) {
                word = cbits[(uint32_t)(bs - first) / 32u + (uint32_t)lane];
                const int avail = kmax - 32 * lane;
                if (avail < 32) word &= (1u << avail) - 1u;
            }
            for (int c = nwords - 1; c >= 0; c--) {
                const uint32_t bits = __shfl_sync(0xffffffffu, word, c);
                const bool set = ((bits >> (31 - lane)) & 1u) != 0u;
                const uint32_t ball = __ballot_sync(0xffffffffu, set);
                if (set) pos[cnt + __popc(ball & lanemask_lt())] = (uint8_t)(32 * c + 31 - lane);
                cnt += __popc(ball);
            }
            __syncwarp();
        }
        for (int gi = 0; gi < cnt; gi += 3) {
            const int ne = min(3, cnt - gi);
            const int k0 = pos[gi], k1 = ne > 1 ? (int)pos[gi + 1] : -1, k2 = ne > 2 ? (int)pos[gi + 2] : -1;
            // unrolled: the three entries' falloff and gradient arithmetic is independent apart
            // from the per-pixel T and gS chain, so the scheduler can overlap it
#pragma unroll
            for (int e = 0; e < 3; e++) {
                if (e >= ne) break;
                const int k = e == 0 ? k0 : (e == 1 ? k1 : k2);
                const float4 e0 = s_e0[k], e1 = s_e1[k], e2 = s_e2[k], e3 = s_e3[k];
                const uint32_t lp = (uint32_t)(bs + k - first);
                float dx;
                float2 dy;
                float2 p = staged_power2(e0, e1, fpx, fpy, &dx, &dy);
                float2 G, nog, na;  // falloff, -o G, -alpha
                if constexpr (EXACT) {
                    // the parity build's decisions: power, G and alpha as the forward took them
                    const float4 cn = s_cn[k];
                    p = make_float2(exact_power(cn, e1.x, e0.x, fpx, fpy.x), exact_power(cn, e1.x, e0.x, fpx, fpy.y));
                    G = make_float2(__double2float_rn(exp((double)p.x)), __double2float_rn(exp((double)p.y)));
                    const float og0 = ieee_mul(cn.w, G.x), og1 = ieee_mul(cn.w, G.y);
                    nog = make_float2(-og0, -og1);
                    na = make_float2(-exact_alpha(og0), -exact_alpha(og1));
                } else {
                    G = make_float2(gauss_exp2(p.x), gauss_exp2(p.y));
                    na = neg_alpha2(e2, G, &nog);
                }
                const bool u0 = lp < nc0 && !(p.x > 0.0f) && !(na.x > nthr);
                const bool u1 = lp < nc1 && !(p.y > 0.0f) && !(na.y > nthr);
                const float2 om = __fadd2_rn(one, na);                 // 1 - alpha
                const float2 inv = make_float2(__fdividef(1.0f, om.x), __fdividef(1.0f, om.y));
                const float2 gc = __ffma2_rn(g2, make_float2(e3.z, e3.w),
                                             __ffma2_rn(g1, make_float2(e3.x, e3.y),
                                                        __fmul2_rn(g0, make_float2(e2.z, e2.w))));
                const float2 dal = __fmul2_rn(inv, __ffma2_rn(gc, T, ngS));  // dL/dalpha
                const float2 Tb = __fmul2_rn(T, inv);                        // T before the entry
                const float2 naT = __fmul2_rn(na, Tb);                       // -alpha T_before
                const float2 ngS2 = __ffma2_rn(naT, gc, ngS);
                T = make_float2(u0 ? Tb.x : T.x, u1 ? Tb.y : T.y);
                ngS = make_float2(u0 ? ngS2.x : ngS.x, u1 ? ngS2.y : ngS.y);
                // the 0.99 clamp passes no gradient to the opacity or the power
                const float2 wG = __fmul2_rn(dal, G);
                const float w0 = (u0 && !(nog.x < -0.99f)) ? wG.x : 0.0f;
                const float w1 = (u1 && !(nog.y < -0.99f)) ? wG.y : 0.0f;
                const float2 nt = make_float2(u0 ? naT.x : 0.0f, u1 ? naT.y : 0.0f);
                const float F = w0 + w1;
                const float2 b = __fmul2_rn(make_float2(w0, w1), dy);
                const float m0 = dx * F, m1 = b.x + b.y;
                const float2 c0g = __fmul2_rn(g0, nt), c1g = __fmul2_rn(g1, nt), c2g = __fmul2_rn(g2, nt);
                red[9 * e + 0][lane] = m0;
                red[9 * e + 1][lane] = m1;
                red[9 * e + 2][lane] = dx * m0;
                red[9 * e + 3][lane] = dx * m1;
                red[9 * e + 4][lane] = fmaf(b.x, dy.x, b.y * dy.y);
                red[9 * e + 5][lane] = F;
                red[9 * e + 6][lane] = c0g.x + c0g.y;
                red[9 * e + 7][lane] = c1g.x + c1g.y;
                red[9 * e + 8][lane] = c2g.x + c2g.y;
                if constexpr (COUNT) pairs += (uint32_t)u0 + (uint32_t)u1;
            }
            __syncwarp();
            if (lane < 9 * ne) {
                const float4* row = reinterpret_cast<const float4*>(red[lane]);
                // the row's 32 values as two packed pairs of running sums
                const float4 r0 = row[0];
                float2 ax = make_float2(r0.x, r0.y), az = make_float2(r0.z, r0.w);
#pragma unroll
                for (int q = 1; q < 8; q++) {
                    const float4 x = row[q];
                    ax = __fadd2_rn(ax, make_float2(x.x, x.y));
                    az = __fadd2_rn(az, make_float2(x.z, x.w));
                }
                const float2 s2 = __fadd2_rn(ax, az);
                const float tot = s2.x + s2.y;
                const int e = lane / 9, comp = lane - 9 * e;
                const int k = e == 0 ? k0 : (e == 1 ? k1 : k2);
                if (tot != 0.0f) atomicAdd(reinterpret_cast<float*>(L.gs) + 12 * (size_t)s_j[k] + comp, tot);
            }
            __syncwarp();
        }
    }
    if constexpr (COUNT) {
        const uint32_t ws = __reduce_add_sync(0xffffffffu, pairs);
        if (lane == 0 && ws) atomicAdd(&L.hdr->pairs_bwd, (unsigned long long)ws);
    }
}

template <int B, int BATCH>
static void bwd_launch(const Layout& L, const uint32_t* tval, const cgs_config& c, const float* dimg, const float* T,
                       const uint32_t* nc, const L1In* l1, cudaStream_t st)
{
    dim3 grid(L.tiles_x, L.tiles_y, L.V);
    const L1In none{};
    const float b0 = c.bg[0], b1 = c.bg[1], b2 = c.bg[2];
    const int NT = B * B / 2;
    if (c.exact) {
        k_render_bwd<B, BATCH, true, 0, true><<<grid, NT, 0, st>>>(L, tval, b0, b1, b2, dimg, T, nc, none);
    } else if (L.count_pairs) {
        if (!l1) k_render_bwd<B, BATCH, false, 0, true><<<grid, NT, 0, st>>>(L, tval, b0, b1, b2, dimg, T, nc, none);
        else if (l1->u8) k_render_bwd<B, BATCH, false, 1, true><<<grid, NT, 0, st>>>(L, tval, b0, b1, b2, nullptr, T, nc, *l1);
        else k_render_bwd<B, BATCH, false, 2, true><<<grid, NT, 0, st>>>(L, tval, b0, b1, b2, nullptr, T, nc, *l1);
    } else {
        if (!l1) k_render_bwd<B, BATCH, false, 0, false><<<grid, NT, 0, st>>>(L, tval, b0, b1, b2, dimg, T, nc, none);
        else if (l1->u8) k_render_bwd<B, BATCH, false, 1, false><<<grid, NT, 0, st>>>(L, tval, b0, b1, b2, nullptr, T, nc, *l1);
        else k_render_bwd<B, BATCH, false, 2, false><<<grid, NT, 0, st>>>(L, tval, b0, b1, b2, nullptr, T, nc, *l1);
    }
}

// l1 != NULL: the L1 loss and its gradient are formed inside the kernel (dimg unused); not
// built for the parity configuration (cgs_config.exact), which then returns false.
bool launch_render_bwd(const Layout& L, const cgs_config& c, const float* dimg, const float* T, const uint32_t* nc,
                       const L1In* l1, cudaStream_t st)
{
    const uint32_t* tv = L.tval;
    if (l1 && c.exact) return false;
    if (L.B == 16) {
        switch (c.batch) {
            case 32: bwd_launch<16, 32>(L, tv, c, dimg, T, nc, l1, st); return true;
            case 64: bwd_launch<16, 64>(L, tv, c, dimg, T, nc, l1, st); return true;
            case 128: bwd_launch<16, 128>(L, tv, c, dimg, T, nc, l1, st); return true;
            case 256: bwd_launch<16, 256>(L, tv, c, dimg, T, nc, l1, st); return true;
        }
    } else if (L.B == 8) {
        switch (c.batch) {
            case 32: bwd_launch<8, 32>(L, tv, c, dimg, T, nc, l1, st); return true;
            case 64: bwd_launch<8, 64>(L, tv, c, dimg, T, nc, l1, st); return true;
        }
    }
    return false;
}

}  // namespace cgs
