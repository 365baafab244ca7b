// Backward of the projection and colour (differentiable rendering, Sec. 3.1): turns the
// per-Gaussian pixel moments accumulated by the compositing backward into the screen-space
// gradients (u, v, conic, opacity, rgb) and chains them to the scene attributes.  Discrete decisions pass no gradient: the
// guard-band clamp zeroes the clamped coordinate's direct term, the colour clamp masks its
// channel, and the quaternion gradient goes through the normalisation.  Compiled with
// -fmad=false like the forward projection, so the recomputed clamp decisions match it.
// Gradients are added with 16-byte vector atomics (one per attribute row).
#include "proj_math.cuh"

namespace cgs {

// Two roles per CTA of 128 threads and 64 visible Gaussians: warps 0-1 chain the geometric
// gradients (u, v, conic, opacity -> mean, scale, rotation), warps 2-3 the colour gradients
// (rgb -> SH coefficients and the view-direction term of the mean).  The split halves the
// registers a thread needs and doubles the threads in flight (registers are further capped
// so six CTAs fit an SM: the kernel is bound by memory latency).  DEG is the scene's SH
// degree, fixed at compile time so the coefficient loops unroll and the per-Gaussian arrays
// live in registers.
//
// Two output forms.  Dense (PACKED false): each role adds its part into gradient arrays laid
// out like the scene (row = scene index) with 16-byte vector atomics, so a Gaussian seen in
// several views of a frame sums its contributions; the caller clears the arrays.  Packed
// (PACKED true): row r of the outputs is the visible list's r-th (view, Gaussian) pair,
// written with plain stores (the two parts of the mean gradient are summed through shared
// memory) together with its scene index; every row below the visible count is written, so
// nothing needs clearing and no gradient line is read back from memory.
constexpr int PB_THREADS = 128;
constexpr int PB_PER_CTA = PB_THREADS / 2;

// Colour role: dL/d(SH coefficient k, channel ch) = Y_k dL/dcolour_ch (clamped channels pass
// nothing) into grow[], and the mean gradient through the view direction into gm_dir.
template <int DEG>
__device__ __forceinline__ void colour_grad(const float m[3], const cgs_camera& c, const cgs_scene& S, long long g,
                                            const float grgb[3], float Yg[48], float gm_dir[3])
{
    constexpr int nc = (DEG + 1) * (DEG + 1);
    float f[48], rgb[3], dir[3], len, Y[16], dY[16][3];
    if (S.attr_fp16) load_sh_half(S.sh, g, nc, f);
    else load_sh(S.sh, g, nc, f);
    const int cl = sh_colour(m, c, f, DEG, rgb, dir, &len, Y);
    sh_grad(dir[0], dir[1], dir[2], DEG, dY);
    float gdir[3] = {0.f, 0.f, 0.f};
    float gc[3];
#pragma unroll
    for (int ch = 0; ch < 3; ch++) gc[ch] = (cl & (1 << ch)) ? 0.0f : grgb[ch];
    // dL/dcolour . f_k per basis function, then through dY_k/d(dir)
#pragma unroll
    for (int k = 0; k < nc; k++) {
        const float fg = f[k * 3] * gc[0] + f[k * 3 + 1] * gc[1] + f[k * 3 + 2] * gc[2];
        gdir[0] += fg * dY[k][0];
        gdir[1] += fg * dY[k][1];
        gdir[2] += fg * dY[k][2];
    }
#pragma unroll
    for (int i = 0; i < nc * 3; i++) Yg[i] = Y[i / 3] * gc[i % 3];
    // the direction's dependence on the mean: d dir / d m = (I - dir dir^T) / len
    const float dd = dir[0] * gdir[0] + dir[1] * gdir[1] + dir[2] * gdir[2];
#pragma unroll
    for (int a = 0; a < 3; a++) gm_dir[a] = (gdir[a] - dir[a] * dd) / len;
}

// Geometry role: (du, dv, dA', dB', dC') of the projected record -> mean, scale and
// rotation gradients (through the quaternion's normalisation), for a successful projection p.
__device__ __forceinline__ void geometry_chain(const Proj& p, const cgs_camera& c, float gu, float gv, float gA_,
                                               float gB_, float gC_, const float s[3], float gm[3], float gsv[3],
                                               float gqn[4])
{
    // conic (C/D, -B/D, A/D), D = AC - B^2 -> Sigma2D entries (A, B, C), over the common
    // denominator D^2 (1/D - AC/D^2 = -B^2/D^2 carries no cancellation this way)
    const float A = p.A, Bv = p.B, C = p.C, D2 = p.det * p.det;
    const float dA = (-gA_ * C * C + gB_ * Bv * C - gC_ * Bv * Bv) / D2;
    const float dB = (2.0f * gA_ * Bv * C - gB_ * (A * C + Bv * Bv) + 2.0f * gC_ * A * Bv) / D2;
    const float dC = (-gA_ * Bv * Bv + gB_ * A * Bv - gC_ * A * A) / D2;

    // Sigma2D = T S T^T
    const float* Tm = p.Tm;
    const float* S3 = p.S3;
    float gS[9];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            gS[a * 3 + b] = dA * Tm[a] * Tm[b] + dB * Tm[a] * Tm[3 + b] + dC * Tm[3 + a] * Tm[3 + b];
    float gT[6];
    for (int a = 0; a < 3; a++) {
        const float st0 = S3[a * 3] * Tm[0] + S3[a * 3 + 1] * Tm[1] + S3[a * 3 + 2] * Tm[2];
        const float st1 = S3[a * 3] * Tm[3] + S3[a * 3 + 1] * Tm[4] + S3[a * 3 + 2] * Tm[5];
        gT[a] = 2.0f * dA * st0 + dB * st1;
        gT[3 + a] = 2.0f * dC * st1 + dB * st0;
    }
    const float* W = c.R;
    float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f;
    for (int a = 0; a < 3; a++) {
        gJ00 += gT[a] * W[a];
        gJ02 += gT[a] * W[6 + a];
        gJ11 += gT[3 + a] * W[3 + a];
        gJ12 += gT[3 + a] * W[6 + a];
    }
    const float fx = c.fx, fy = c.fy, tx = p.tx, ty = p.ty, tz = p.tz;
    const float tz2 = tz * tz, tz3 = tz2 * tz;
    float gtx = 0.f, gty = 0.f, gtz = 0.f;
    gtz += gJ00 * (-fx / tz2) + gJ11 * (-fy / tz2);
    if (!p.clampx) { gtx += gJ02 * (-fx / tz2); gtz += gJ02 * (2.0f * fx * tx / tz3); }
    else { const float lim = tx / tz > 0.f ? p.limx : -p.limx; gtz += gJ02 * (fx * lim / tz2); }
    if (!p.clampy) { gty += gJ12 * (-fy / tz2); gtz += gJ12 * (2.0f * fy * ty / tz3); }
    else { const float lim = ty / tz > 0.f ? p.limy : -p.limy; gtz += gJ12 * (fy * lim / tz2); }
    gtx += gu * fx / tz;
    gtz += gu * (-fx * tx / tz2);
    gty += gv * fy / tz;
    gtz += gv * (-fy * ty / tz2);
    for (int a = 0; a < 3; a++) gm[a] = W[a] * gtx + W[3 + a] * gty + W[6 + a] * gtz;

    // Sigma3D = M M^T, M = Rq diag(s)
    float gM[9];
    for (int a = 0; a < 3; a++)
        for (int k = 0; k < 3; k++) {
            float acc = 0.f;
            for (int b = 0; b < 3; b++) acc += (gS[a * 3 + b] + gS[b * 3 + a]) * p.M[b * 3 + k];
            gM[a * 3 + k] = acc;
        }
    float gR[9];
    for (int k = 0; k < 3; k++) {
        float acc = 0.f;
        for (int a = 0; a < 3; a++) acc += gM[a * 3 + k] * p.Rq[a * 3 + k];
        gsv[k] = acc;
        for (int a = 0; a < 3; a++) gR[a * 3 + k] = gM[a * 3 + k] * s[k];
    }
    const float w = p.qn[0], x = p.qn[1], y = p.qn[2], z = p.qn[3];
    float gq[4];
    gq[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gq[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] - 2.f * x * gR[8]);
    gq[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] - 2.f * y * gR[8]);
    gq[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] + x * gR[6] + y * gR[7]);
    const float qd = w * gq[0] + x * gq[1] + y * gq[2] + z * gq[3];
    const float il = 1.0f / p.qlen;
    for (int a = 0; a < 4; a++) gqn[a] = (gq[a] - p.qn[a] * qd) * il;
}

template <int DEG, bool PACKED>
__global__ void __launch_bounds__(PB_THREADS, 6) k_project_bwd(Layout L, cgs_scene S, const cgs_camera* __restrict__ cams,
                                                            float near_z, float* __restrict__ g_mo,
                                                            float* __restrict__ g_sc, float* __restrict__ g_q,
                                                            float* __restrict__ g_sh, long long* __restrict__ g_index)
{
    __shared__ float s_cm[3][PB_PER_CTA];  // packed form: the colour role's mean term
    // over the compacted visible Gaussians, so every lane has work
    const uint32_t n = L.hdr->n_vis;
    const uint32_t* __restrict__ vis = L.vis;
    constexpr int nc = (DEG + 1) * (DEG + 1);
    const bool colour_role = threadIdx.x >= PB_PER_CTA;
    const uint32_t li = threadIdx.x - (colour_role ? PB_PER_CTA : 0);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t stride = gridDim.x * PB_PER_CTA;
    for (uint32_t r0 = blockIdx.x * PB_PER_CTA; r0 < n; r0 += stride) {
        const uint32_t r = r0 + li;
        const bool valid = r < n;
        const uint32_t j = valid ? vis[r] : 0u;
        // the visible-list slot of this thread's next Gaussian, read now and used at the end of
        // the iteration to fetch that Gaussian's rows into L2
        const bool more = r + stride < n;
        const uint32_t jn = more ? vis[r + stride] : 0u;
        float4 ga = z4, gb = z4, gc4 = z4;
        if (valid) {
            ga = L.gs[3 * (size_t)j];
            gb = L.gs[3 * (size_t)j + 1];
            gc4 = L.gs[3 * (size_t)j + 2];
        }
        __syncthreads();  // both roles have read the accumulators; clear them (no forward does: each
                          // backward leaves every row the compositing backward added to at zero)
        float gm[3] = {0.f, 0.f, 0.f}, gsv[3] = {0.f, 0.f, 0.f}, gqn[4] = {0.f, 0.f, 0.f, 0.f};
        long long g = 0;
        if (valid) {
            if (!colour_role) {
                L.gs[3 * (size_t)j] = z4;
                L.gs[3 * (size_t)j + 1] = z4;
            } else {
                L.gs[3 * (size_t)j + 2] = z4;
            }
            const int v = (int)(L.pkey[j] >> 32);
            g = L.gidx[j];
            const cgs_camera& c = cams[v];
            const float4 mo = __ldg(reinterpret_cast<const float4*>(S.mean_opac) + g);
            const float m[3] = {mo.x, mo.y, mo.z};
            if (colour_role) {
                // the accumulated colour moments are the negated colour gradient
                const float grgb[3] = {-gb.z, -gb.w, -gc4.x};
                float Yg[48];
                colour_grad<DEG>(m, c, S, g, grgb, Yg, gm);
                float* gsh = g_sh + (PACKED ? (long long)r : g) * (long long)(nc * 3);
                if constexpr ((nc * 3) % 4 == 0) {
                    float4* g4 = reinterpret_cast<float4*>(gsh);
#pragma unroll
                    for (int i = 0; i < nc * 3 / 4; i++) {
                        const float4 x = make_float4(Yg[4 * i], Yg[4 * i + 1], Yg[4 * i + 2], Yg[4 * i + 3]);
                        if (PACKED) g4[i] = x;
                        else atomicAdd(g4 + i, x);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < nc * 3; i++) {
                        if (PACKED) gsh[i] = Yg[i];
                        else atomicAdd(gsh + i, Yg[i]);
                    }
                }
                if (PACKED) {
                    s_cm[0][li] = gm[0];
                    s_cm[1][li] = gm[1];
                    s_cm[2][li] = gm[2];
                } else {
                    atomicAdd(reinterpret_cast<float4*>(g_mo) + g, make_float4(gm[0], gm[1], gm[2], 0.0f));
                }
            } else {
                float s[3], q[4];
                load_scale_quat(S, g, s, q);
                Proj p;
                if (project_one(m, s, q, c, near_z, p) == 0) {
                    // the pixel moments of w = dL/do (m0..m4 in ga.xyzw, gb.x): dL/dpower = o w
                    // and power = -A'/2 dx^2 - B' dx dy - C'/2 dy^2 with dx = u - px
                    const float o = mo.w;
                    const float mx = o * ga.x, my = o * ga.y;
                    const float gu = -(p.conic[0] * mx + p.conic[1] * my);
                    const float gv = -(p.conic[2] * my + p.conic[1] * mx);
                    geometry_chain(p, c, gu, gv, -0.5f * o * ga.z, -o * ga.w, -0.5f * o * gb.x, s, gm, gsv, gqn);
                }
                const long long row = PACKED ? (long long)r : g;
                const float4 x_sc = make_float4(gsv[0], gsv[1], gsv[2], 0.0f);
                const float4 x_q = make_float4(gqn[0], gqn[1], gqn[2], gqn[3]);
                if (PACKED) {
                    reinterpret_cast<float4*>(g_sc)[row] = x_sc;
                    reinterpret_cast<float4*>(g_q)[row] = x_q;
                    g_index[row] = g;
                } else {
                    atomicAdd(reinterpret_cast<float4*>(g_mo) + row, make_float4(gm[0], gm[1], gm[2], gb.y));
                    atomicAdd(reinterpret_cast<float4*>(g_sc) + row, x_sc);
                    atomicAdd(reinterpret_cast<float4*>(g_q) + row, x_q);
                }
            }
        }
        if (PACKED) {
            __syncthreads();  // the colour role's mean terms are in shared memory
            if (valid && !colour_role)
                reinterpret_cast<float4*>(g_mo)[r] =
                    make_float4(gm[0] + s_cm[0][li], gm[1] + s_cm[1][li], gm[2] + s_cm[2][li], gb.y);
        }
        if (more) {
            // the next Gaussian's rows into L2: the accumulator row and the attribute rows this
            // role reads
            const long long gn = L.gidx[jn];
            const char* acc = reinterpret_cast<const char*>(L.gs + 3 * (size_t)jn);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(acc));
            if (colour_role) {
                const size_t row = (size_t)(nc * 3) * (S.attr_fp16 ? 2u : 4u);
                const char* q = reinterpret_cast<const char*>(S.sh) + (size_t)gn * row;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
                if (row > 64) asm volatile("prefetch.global.L2 [%0];" ::"l"(q + row - 1));
            } else {
                const size_t ab = S.attr_fp16 ? 8u : 16u;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(S.mean_opac) + 16 * (size_t)gn));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(S.scale) + ab * (size_t)gn));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(S.quat) + ab * (size_t)gn));
            }
        }
    }
}

void launch_project_bwd(const Layout& L, const cgs_scene& S, const cgs_camera* cams, float near_z, float* g_mo,
                        float* g_sc, float* g_q, float* g_sh, long long* g_index, int n_sm, cudaStream_t st)
{
    // one wave of resident CTAs (six per SM); each loops over the visible list, fetching its
    // next Gaussian's rows into L2 while it works on the current one
    long long want = (L.n_cap + PB_PER_CTA - 1) / PB_PER_CTA;
    long long grid = want < (long long)n_sm * 6 ? want : (long long)n_sm * 6;
    if (grid < 1) grid = 1;
    const unsigned gr = (unsigned)grid;
#define CGS_PB_LAUNCH(D)                                                                                  \
    if (g_index) k_project_bwd<D, true><<<gr, PB_THREADS, 0, st>>>(L, S, cams, near_z, g_mo, g_sc, g_q, g_sh, g_index); \
    else k_project_bwd<D, false><<<gr, PB_THREADS, 0, st>>>(L, S, cams, near_z, g_mo, g_sc, g_q, g_sh, nullptr)
    switch (S.sh_degree) {
        case 0: CGS_PB_LAUNCH(0); break;
        case 1: CGS_PB_LAUNCH(1); break;
        case 2: CGS_PB_LAUNCH(2); break;
        default: CGS_PB_LAUNCH(3); break;
    }
#undef CGS_PB_LAUNCH
}

}  // namespace cgs
