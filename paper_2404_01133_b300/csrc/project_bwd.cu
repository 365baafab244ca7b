// Backward of the projection and colour (differentiable rendering, Sec. 3.1): chains the
// per-Gaussian screen-space gradients (u, v, conic, opacity, rgb) accumulated by the
// compositing backward to the scene attributes.  Discrete decisions pass no gradient: the
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
// so six CTAs fit an SM: the kernel is bound by memory latency); each role adds its own part
// of the mean gradient.  DEG is the scene's SH degree, fixed at compile time so the coefficient
// loops unroll and the per-Gaussian arrays live in registers.
constexpr int PB_THREADS = 128;
constexpr int PB_PER_CTA = PB_THREADS / 2;

template <int DEG>
__global__ void __launch_bounds__(PB_THREADS, 6) k_project_bwd(Layout L, cgs_scene S, const cgs_camera* __restrict__ cams,
                                                            float near_z, float* __restrict__ g_mo,
                                                            float* __restrict__ g_sc, float* __restrict__ g_q,
                                                            float* __restrict__ g_sh)
{
    // over the compacted visible Gaussians, so every lane has work
    const uint32_t n = L.hdr->n_vis;
    const uint32_t* __restrict__ vis = L.vis;
    constexpr int deg = DEG;
    constexpr int nc = (DEG + 1) * (DEG + 1);
    const bool colour_role = threadIdx.x >= PB_PER_CTA;
    const uint32_t li = threadIdx.x - (colour_role ? PB_PER_CTA : 0);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t r0 = blockIdx.x * PB_PER_CTA; r0 < n; r0 += gridDim.x * PB_PER_CTA) {
        const uint32_t r = r0 + li;
        const bool valid = r < n;
        const uint32_t j = valid ? vis[r] : 0u;
        float4 ga = z4, gb = z4, gc4 = z4;
        if (valid) {
            ga = L.gs[3 * (size_t)j];
            gb = L.gs[3 * (size_t)j + 1];
            gc4 = L.gs[3 * (size_t)j + 2];
        }
        __syncthreads();  // both roles have read the accumulators; clear them for the next backward
        if (valid) {
            if (!colour_role) {
                L.gs[3 * (size_t)j] = z4;
                L.gs[3 * (size_t)j + 1] = z4;
            } else {
                L.gs[3 * (size_t)j + 2] = z4;
            }
        }
        if (!valid) continue;
        const int v = (int)(L.pkey[j] >> 32);
        const long long g = L.gidx[j];
        const cgs_camera c = cams[v];
        const float4 mo = __ldg(reinterpret_cast<const float4*>(S.mean_opac) + g);
        const float m[3] = {mo.x, mo.y, mo.z};
        if (colour_role) {
            // colour -> SH coefficients and the view direction
            const float grgb[3] = {gb.z, gb.w, gc4.x};
            float f[48], rgb[3], dir[3], len, Y[16], dY[16][3];
            if (S.attr_fp16) load_sh_half(S.sh, g, nc, f);
            else load_sh(S.sh, g, nc, f);
            const int cl = sh_colour(m, c, f, deg, rgb, dir, &len, Y);
            sh_grad(dir[0], dir[1], dir[2], deg, dY);
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
            // dL/df_k = Y_k dL/dcolour, added 16 bytes at a time
            float* gsh = g_sh + g * (long long)(nc * 3);
            if constexpr ((nc * 3) % 4 == 0) {
                float4* g4 = reinterpret_cast<float4*>(gsh);
#pragma unroll
                for (int i = 0; i < nc * 3 / 4; i++)
                    atomicAdd(g4 + i, make_float4(Y[(4 * i) / 3] * gc[(4 * i) % 3],
                                                  Y[(4 * i + 1) / 3] * gc[(4 * i + 1) % 3],
                                                  Y[(4 * i + 2) / 3] * gc[(4 * i + 2) % 3],
                                                  Y[(4 * i + 3) / 3] * gc[(4 * i + 3) % 3]));
            } else {
#pragma unroll
                for (int i = 0; i < nc * 3; i++) atomicAdd(gsh + i, Y[i / 3] * gc[i % 3]);
            }
            // the direction's dependence on the mean: d dir / d m = (I - dir dir^T) / len
            const float dd = dir[0] * gdir[0] + dir[1] * gdir[1] + dir[2] * gdir[2];
            atomicAdd(reinterpret_cast<float4*>(g_mo) + g,
                      make_float4((gdir[0] - dir[0] * dd) / len, (gdir[1] - dir[1] * dd) / len,
                                  (gdir[2] - dir[2] * dd) / len, 0.0f));
            continue;
        }
        const float gu = ga.x, gv = ga.y, gA_ = ga.z, gB_ = ga.w, gC_ = gb.x, gop = gb.y;
        float s[3], q[4];
        load_scale_quat(S, g, s, q);
        Proj p;
        if (project_one(m, s, q, c, near_z, p) != 0) continue;
        float gm[3] = {0.f, 0.f, 0.f};
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
        atomicAdd(reinterpret_cast<float4*>(g_mo) + g, make_float4(gm[0], gm[1], gm[2], gop));

        // Sigma3D = M M^T, M = Rq diag(s)
        float gM[9];
        for (int a = 0; a < 3; a++)
            for (int k = 0; k < 3; k++) {
                float acc = 0.f;
                for (int b = 0; b < 3; b++) acc += (gS[a * 3 + b] + gS[b * 3 + a]) * p.M[b * 3 + k];
                gM[a * 3 + k] = acc;
            }
        float gR[9], gsv[3];
        for (int k = 0; k < 3; k++) {
            float acc = 0.f;
            for (int a = 0; a < 3; a++) acc += gM[a * 3 + k] * p.Rq[a * 3 + k];
            gsv[k] = acc;
            for (int a = 0; a < 3; a++) gR[a * 3 + k] = gM[a * 3 + k] * s[k];
        }
        atomicAdd(reinterpret_cast<float4*>(g_sc) + g, make_float4(gsv[0], gsv[1], gsv[2], 0.0f));
        const float w = p.qn[0], x = p.qn[1], y = p.qn[2], z = p.qn[3];
        float gq[4];
        gq[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
        gq[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] - 2.f * x * gR[8]);
        gq[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] - 2.f * y * gR[8]);
        gq[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] + x * gR[6] + y * gR[7]);
        const float qd = w * gq[0] + x * gq[1] + y * gq[2] + z * gq[3];
        const float il = 1.0f / p.qlen;
        atomicAdd(reinterpret_cast<float4*>(g_q) + g,
                  make_float4((gq[0] - p.qn[0] * qd) * il, (gq[1] - p.qn[1] * qd) * il, (gq[2] - p.qn[2] * qd) * il,
                              (gq[3] - p.qn[3] * qd) * il));
    }
}

void launch_project_bwd(const Layout& L, const cgs_scene& S, const cgs_camera* cams, float near_z, float* g_mo,
                        float* g_sc, float* g_q, float* g_sh, int n_sm, cudaStream_t st)
{
    long long want = (L.n_cap + PB_PER_CTA - 1) / PB_PER_CTA;
    long long grid = want < (long long)n_sm * 16 ? want : (long long)n_sm * 16;
    if (grid < 1) grid = 1;
    switch (S.sh_degree) {
        case 0: k_project_bwd<0><<<(unsigned)grid, PB_THREADS, 0, st>>>(L, S, cams, near_z, g_mo, g_sc, g_q, g_sh); break;
        case 1: k_project_bwd<1><<<(unsigned)grid, PB_THREADS, 0, st>>>(L, S, cams, near_z, g_mo, g_sc, g_q, g_sh); break;
        case 2: k_project_bwd<2><<<(unsigned)grid, PB_THREADS, 0, st>>>(L, S, cams, near_z, g_mo, g_sc, g_q, g_sh); break;
        default: k_project_bwd<3><<<(unsigned)grid, PB_THREADS, 0, st>>>(L, S, cams, near_z, g_mo, g_sc, g_q, g_sh); break;
    }
}

}  // namespace cgs
