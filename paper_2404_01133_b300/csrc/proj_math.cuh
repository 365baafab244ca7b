// Per-Gaussian projection proj(G_k, kappa, tau_i) of Eq. 1 (Sec. 3.1) with the EWA
// splatting conventions the paper defers to its 3DGS citation, plus SH colour.
//
// Every expression is written in a fixed evaluation order.  The forward projection is
// compiled with -fmad=false, IEEE division and square root, so the values that decide
// integers (culls, radius, tile rect, depth bits) are reproducible bit for bit by any
// FP32 implementation that evaluates the same expressions in the same order.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace cgs {

struct Proj {
    float tx, ty, tz;
    float limx, limy;
    bool clampx, clampy;
    float J00, J02, J11, J12;
    float Tm[6];         // T = J W, rows 0 and 1
    float qn[4], qlen;
    float Rq[9];
    float M[9];          // Rq diag(s)
    float S3[9];         // Sigma3D = M M^T
    float A, B, C, det;  // Sigma2D + 0.3 on the diagonal
    float conic[3];
    float u, v, lam1;
};

// Steps 1-6.  Returns 0 visible, 1 behind the near plane, 2 degenerate covariance.
__device__ __forceinline__ int project_one(const float m[3], const float s[3], const float q[4],
                                           const cgs_camera& c, float near_z, Proj& p)
{
    const float* R = c.R;
    p.tx = ((R[0] * m[0] + R[1] * m[1]) + R[2] * m[2]) + c.t[0];
    p.ty = ((R[3] * m[0] + R[4] * m[1]) + R[5] * m[2]) + c.t[1];
    p.tz = ((R[6] * m[0] + R[7] * m[1]) + R[8] * m[2]) + c.t[2];
    p.clampx = p.clampy = false;
    if (!(p.tz > near_z)) return 1;

    const float Wf = (float)c.width, Hf = (float)c.height;
    p.limx = 1.3f * ((0.5f * Wf) / c.fx);
    p.limy = 1.3f * ((0.5f * Hf) / c.fy);
    float xz = p.tx / p.tz, yz = p.ty / p.tz;
    float xzc = xz, yzc = yz;
    if (xz > p.limx) { xzc = p.limx; p.clampx = true; }
    if (xz < -p.limx) { xzc = -p.limx; p.clampx = true; }
    if (yz > p.limy) { yzc = p.limy; p.clampy = true; }
    if (yz < -p.limy) { yzc = -p.limy; p.clampy = true; }
    float txc = xzc * p.tz, tyc = yzc * p.tz;
    float tz2 = p.tz * p.tz;
    p.J00 = c.fx / p.tz;
    p.J02 = -(c.fx * txc) / tz2;
    p.J11 = c.fy / p.tz;
    p.J12 = -(c.fy * tyc) / tz2;

    p.qlen = sqrtf(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
#pragma unroll
    for (int i = 0; i < 4; i++) p.qn[i] = q[i] / p.qlen;
    const float w = p.qn[0], x = p.qn[1], y = p.qn[2], z = p.qn[3];
    p.Rq[0] = 1.0f - 2.0f * (y * y + z * z);
    p.Rq[1] = 2.0f * (x * y - w * z);
    p.Rq[2] = 2.0f * (x * z + w * y);
    p.Rq[3] = 2.0f * (x * y + w * z);
    p.Rq[4] = 1.0f - 2.0f * (x * x + z * z);
    p.Rq[5] = 2.0f * (y * z - w * x);
    p.Rq[6] = 2.0f * (x * z - w * y);
    p.Rq[7] = 2.0f * (y * z + w * x);
    p.Rq[8] = 1.0f - 2.0f * (x * x + y * y);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) p.M[i * 3 + k] = p.Rq[i * 3 + k] * s[k];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            p.S3[i * 3 + j] = (p.M[i * 3 + 0] * p.M[j * 3 + 0] + p.M[i * 3 + 1] * p.M[j * 3 + 1])
                              + p.M[i * 3 + 2] * p.M[j * 3 + 2];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        p.Tm[j] = p.J00 * R[j] + p.J02 * R[6 + j];
        p.Tm[3 + j] = p.J11 * R[3 + j] + p.J12 * R[6 + j];
    }
    float U[6];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            U[a * 3 + j] = (p.Tm[a * 3 + 0] * p.S3[j] + p.Tm[a * 3 + 1] * p.S3[3 + j]) + p.Tm[a * 3 + 2] * p.S3[6 + j];
    float s00 = (U[0] * p.Tm[0] + U[1] * p.Tm[1]) + U[2] * p.Tm[2];
    float s01 = (U[0] * p.Tm[3] + U[1] * p.Tm[4]) + U[2] * p.Tm[5];
    float s11 = (U[3] * p.Tm[3] + U[4] * p.Tm[4]) + U[5] * p.Tm[5];
    p.A = s00 + 0.3f;
    p.B = s01;
    p.C = s11 + 0.3f;
    p.det = p.A * p.C - p.B * p.B;
    if (!(p.det > 0.0f)) return 2;
    p.conic[0] = p.C / p.det;
    p.conic[1] = -p.B / p.det;
    p.conic[2] = p.A / p.det;
    float mid = 0.5f * (p.A + p.C);
    float disc = mid * mid - p.det;
    float root = sqrtf(disc > 0.1f ? disc : 0.1f);
    float l1 = mid + root, l2 = mid - root;
    p.lam1 = l1 > l2 ? l1 : l2;
    p.u = (c.fx * p.tx) / p.tz + c.cx;
    p.v = (c.fy * p.ty) / p.tz + c.cy;
    return 0;
}

// Real SH constants (orthonormal, Condon-Shortley phase), correctly rounded to FP32.
#define SH_K0 2.820948064e-01f
#define SH_K1 4.886025190e-01f
#define SH_K2 1.092548490e+00f
#define SH_K3 3.153915703e-01f
#define SH_K4 5.462742448e-01f
#define SH_K5 5.900436044e-01f
#define SH_K6 2.890611410e+00f
#define SH_K7 4.570457935e-01f
#define SH_K8 3.731763363e-01f
#define SH_K9 1.445305705e+00f

// Basis Y[0..nc) at the unit direction (x, y, z), index l^2 + l + m.
__device__ __forceinline__ void sh_eval(float x, float y, float z, int deg, float Y[16])
{
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    Y[0] = SH_K0;
    if (deg < 1) return;
    Y[1] = -SH_K1 * y;
    Y[2] = SH_K1 * z;
    Y[3] = -SH_K1 * x;
    if (deg < 2) return;
    Y[4] = SH_K2 * xy;
    Y[5] = -SH_K2 * yz;
    Y[6] = SH_K3 * ((2.0f * zz - xx) - yy);
    Y[7] = -SH_K2 * xz;
    Y[8] = SH_K4 * (xx - yy);
    if (deg < 3) return;
    Y[9] = (-SH_K5 * y) * (3.0f * xx - yy);
    Y[10] = SH_K6 * (xy * z);
    Y[11] = (-SH_K7 * y) * ((4.0f * zz - xx) - yy);
    Y[12] = (SH_K8 * z) * ((2.0f * zz - 3.0f * xx) - 3.0f * yy);
    Y[13] = (-SH_K7 * x) * ((4.0f * zz - xx) - yy);
    Y[14] = (SH_K9 * z) * (xx - yy);
    Y[15] = (-SH_K5 * x) * (xx - 3.0f * yy);
}

// Partial derivatives of the basis polynomials in x, y, z.
__device__ __forceinline__ void sh_grad(float x, float y, float z, int deg, float dY[16][3])
{
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
#pragma unroll
    for (int k = 0; k < 16; k++) dY[k][0] = dY[k][1] = dY[k][2] = 0.0f;
    if (deg < 1) return;
    dY[1][1] = -SH_K1;
    dY[2][2] = SH_K1;
    dY[3][0] = -SH_K1;
    if (deg < 2) return;
    dY[4][0] = SH_K2 * y;  dY[4][1] = SH_K2 * x;
    dY[5][1] = -SH_K2 * z; dY[5][2] = -SH_K2 * y;
    dY[6][0] = SH_K3 * (-2.0f * x); dY[6][1] = SH_K3 * (-2.0f * y); dY[6][2] = SH_K3 * (4.0f * z);
    dY[7][0] = -SH_K2 * z; dY[7][2] = -SH_K2 * x;
    dY[8][0] = SH_K4 * (2.0f * x); dY[8][1] = SH_K4 * (-2.0f * y);
    if (deg < 3) return;
    dY[9][0] = -SH_K5 * (6.0f * xy);          dY[9][1] = -SH_K5 * (3.0f * xx - 3.0f * yy);
    dY[10][0] = SH_K6 * yz;                   dY[10][1] = SH_K6 * xz; dY[10][2] = SH_K6 * xy;
    dY[11][0] = -SH_K7 * (-2.0f * xy);        dY[11][1] = -SH_K7 * ((4.0f * zz - xx) - 3.0f * yy);
    dY[11][2] = -SH_K7 * (8.0f * yz);
    dY[12][0] = SH_K8 * (-6.0f * xz);         dY[12][1] = SH_K8 * (-6.0f * yz);
    dY[12][2] = SH_K8 * ((6.0f * zz - 3.0f * xx) - 3.0f * yy);
    dY[13][0] = -SH_K7 * ((4.0f * zz - 3.0f * xx) - yy); dY[13][1] = -SH_K7 * (-2.0f * xy);
    dY[13][2] = -SH_K7 * (8.0f * xz);
    dY[14][0] = SH_K9 * (2.0f * xz);          dY[14][1] = SH_K9 * (-2.0f * yz); dY[14][2] = SH_K9 * (xx - yy);
    dY[15][0] = -SH_K5 * (3.0f * xx - 3.0f * yy); dY[15][1] = -SH_K5 * (-6.0f * xy);
}

__device__ __forceinline__ float h2f(unsigned short b) { return __half2float(__ushort_as_half(b)); }

// Scale and rotation of Gaussian g, FP32 or FP16 storage (exact conversion to FP32).
__device__ __forceinline__ void load_scale_quat(const cgs_scene& S, long long g, float s[3], float q[4])
{
    if (S.attr_fp16) {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(S.scale) + g);
        const uint2 b = __ldg(reinterpret_cast<const uint2*>(S.quat) + g);
        s[0] = h2f(a.x & 0xffffu); s[1] = h2f(a.x >> 16); s[2] = h2f(a.y & 0xffffu);
        q[0] = h2f(b.x & 0xffffu); q[1] = h2f(b.x >> 16); q[2] = h2f(b.y & 0xffffu); q[3] = h2f(b.y >> 16);
    } else {
        const float4 a = __ldg(reinterpret_cast<const float4*>(S.scale) + g);
        const float4 b = __ldg(reinterpret_cast<const float4*>(S.quat) + g);
        s[0] = a.x; s[1] = a.y; s[2] = a.z;
        q[0] = b.x; q[1] = b.y; q[2] = b.z; q[3] = b.w;
    }
}

// Loads the nc*3 SH coefficients of Gaussian g from FP16 storage.
__device__ __forceinline__ void load_sh_half(const void* __restrict__ shv, long long g, int nc, float f[48])
{
    const unsigned short* src = reinterpret_cast<const unsigned short*>(shv) + g * (long long)(nc * 3);
    if (nc == 16) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
        for (int i = 0; i < 6; i++) {
            const uint4 v = __ldg(s4 + i);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                f[8 * i + 2 * k] = h2f(w[k] & 0xffffu);
                f[8 * i + 2 * k + 1] = h2f(w[k] >> 16);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < nc * 3; i++) f[i] = h2f(__ldg(src + i));
    }
}

// Loads the nc*3 SH coefficients of Gaussian g (contiguous, channel fastest).
__device__ __forceinline__ void load_sh(const float* __restrict__ sh, long long g, int nc, float f[48])
{
    const float* src = sh + g * (long long)(nc * 3);
    if (nc == 16) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int i = 0; i < 12; i++) {
            float4 v = __ldg(s4 + i);
            f[4 * i] = v.x; f[4 * i + 1] = v.y; f[4 * i + 2] = v.z; f[4 * i + 3] = v.w;
        }
    } else if (nc == 4) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int i = 0; i < 3; i++) {
            float4 v = __ldg(s4 + i);
            f[4 * i] = v.x; f[4 * i + 1] = v.y; f[4 * i + 2] = v.z; f[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < nc * 3; i++) f[i] = __ldg(src + i);
    }
}

// View direction and colour: raw = sum_k Y_k f_k + 0.5 (k ascending), clamped at 0.
// Returns a 3-bit mask of clamped channels.
__device__ __forceinline__ int sh_colour(const float m[3], const cgs_camera& c, const float* f, int deg,
                                         float rgb[3], float dir[3], float* len_out, float Y[16])
{
    float d0 = m[0] - c.campos[0], d1 = m[1] - c.campos[1], d2 = m[2] - c.campos[2];
    float len = sqrtf((d0 * d0 + d1 * d1) + d2 * d2);
    dir[0] = d0 / len; dir[1] = d1 / len; dir[2] = d2 / len;
    *len_out = len;
    sh_eval(dir[0], dir[1], dir[2], deg, Y);
    const int nc = (deg + 1) * (deg + 1);
    int clamp = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        float acc = Y[0] * f[ch];
#pragma unroll
        for (int k = 1; k < nc; k++) acc = acc + Y[k] * f[k * 3 + ch];
        acc = acc + 0.5f;
        if (acc < 0.0f) { rgb[ch] = 0.0f; clamp |= 1 << ch; }
        else rgb[ch] = acc;
    }
    return clamp;
}

// sh_colour with the coefficients read from the scene in chunks of four basis functions (12
// values, three 16-byte loads issued together) instead of staged all at once in registers:
// the same operations in the same order, so the same colour bit for bit, in far fewer
// registers, with one memory latency per chunk rather than per coefficient.
template <int DEG>
__device__ __forceinline__ void sh_colour_streamed(const float m[3], const cgs_camera& c, const cgs_scene& S,
                                                   long long g, float rgb[3])
{
    constexpr int nc = (DEG + 1) * (DEG + 1);
    constexpr int nchunk = (nc + 3) / 4;
    const float d0 = m[0] - c.campos[0], d1 = m[1] - c.campos[1], d2 = m[2] - c.campos[2];
    const float len = sqrtf((d0 * d0 + d1 * d1) + d2 * d2);
    float Y[16];
    sh_eval(d0 / len, d1 / len, d2 / len, DEG, Y);
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int ck = 0; ck < nchunk; ck++) {
        float f[12];
        constexpr int per = 12;
        const int k0 = 4 * ck;
        const int cnt = (nc - k0) < 4 ? 3 * (nc - k0) : per;  // values in this chunk
        if (S.attr_fp16) {
            const unsigned short* src = reinterpret_cast<const unsigned short*>(S.sh) + g * (long long)(nc * 3) + 3 * k0;
            if (nc == 16) {
                const uint2* s2 = reinterpret_cast<const uint2*>(src);  // 24-byte aligned rows: 8-byte loads
                const uint2 u0 = __ldg(s2), u1 = __ldg(s2 + 1), u2 = __ldg(s2 + 2);
                const uint32_t w[6] = {u0.x, u0.y, u1.x, u1.y, u2.x, u2.y};
#pragma unroll
                for (int i = 0; i < 6; i++) {
                    f[2 * i] = h2f(w[i] & 0xffffu);
                    f[2 * i + 1] = h2f(w[i] >> 16);
                }
            } else {
#pragma unroll
                for (int i = 0; i < per; i++) f[i] = i < cnt ? h2f(__ldg(src + i)) : 0.0f;
            }
        } else {
            const float* src = S.sh + g * (long long)(nc * 3) + 3 * k0;
            if (nc == 16 || nc == 4) {
                const float4* s4 = reinterpret_cast<const float4*>(src);
                const float4 a = __ldg(s4), b = __ldg(s4 + 1), cc = __ldg(s4 + 2);
                f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
                f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
                f[8] = cc.x; f[9] = cc.y; f[10] = cc.z; f[11] = cc.w;
            } else {
#pragma unroll
                for (int i = 0; i < per; i++) f[i] = i < cnt ? __ldg(src + i) : 0.0f;
            }
        }
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            const int k = k0 + kk;
            if (k >= nc) break;
#pragma unroll
            for (int ch = 0; ch < 3; ch++)
                acc[ch] = k == 0 ? Y[0] * f[ch] : acc[ch] + Y[k] * f[3 * kk + ch];
        }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        const float v = acc[ch] + 0.5f;
        rgb[ch] = v < 0.0f ? 0.0f : v;
    }
}

// Maps a flattened selected index j to (view, scene index) through the per-view segment
// lists built by the selection kernel (binary searches over short prefix arrays).
__device__ __forceinline__ void locate(const Layout& L, uint32_t j, int* view_out, long long* g_out)
{
    int lo = 0, hi = L.V;  // view_base[lo] <= j < view_base[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (L.view_base[mid] <= j) lo = mid; else hi = mid;
    }
    const int v = lo;
    const uint32_t i = j - L.view_base[v];
    const uint32_t* sb = L.seg_base + (size_t)v * (L.NB + 1);
    int s0 = 0, s1 = (int)L.n_seg[v];
    while (s1 - s0 > 1) {
        int mid = (s0 + s1) >> 1;
        if (sb[mid] <= i) s0 = mid; else s1 = mid;
    }
    *view_out = v;
    *g_out = L.seg_off[(size_t)v * L.NB + s0] + (long long)(i - sb[s0]);
}

// Block of the selected index j and its rank inside the block's segment (segment of `view`).
__device__ __forceinline__ void locate_block(const Layout& L, uint32_t j, int v, int* blk, uint32_t* rank)
{
    const uint32_t i = j - L.view_base[v];
    const uint32_t* sb = L.seg_base + (size_t)v * (L.NB + 1);
    int s0 = 0, s1 = (int)L.n_seg[v];
    while (s1 - s0 > 1) {
        int mid = (s0 + s1) >> 1;
        if (sb[mid] <= i) s0 = mid; else s1 = mid;
    }
    *blk = L.seg_blk[(size_t)v * L.NB + s0];
    *rank = i - sb[s0];
}

}  // namespace cgs
