// Shared pieces of the compositing kernels (stage d of the hot path: Eq. 1, Sec. 3.1, and its
// backward replay): the per-pair power and exponential, the staged-entry layout and the packed
// pair arithmetic of a lane's two pixels, and the per-warp culling masks.
//
// One CTA per (view, tile), two pixels per thread.  Each round stages `BATCH` projected
// records of the tile's depth-sorted list in shared memory; a pixel blends with
// alpha = min(0.99, o exp(power)), skips alpha < 1/255 and stops before the entry that
// would take its transmittance below 1e-4.
#pragma once

#include "common.cuh"

namespace cgs {

// Every operation of the per-pair power is written as an explicit IEEE instruction in PTX
// (round to nearest, denormals kept), so the forward and the backward kernels compute the same
// bits whatever their translation units' floating-point flags (the backward is built with
// flush-to-zero) and take identical skip and stop decisions.
__device__ __forceinline__ float ieee_sub(float a, float b)
{
    float r;
    asm("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float ieee_add(float a, float b)
{
    float r;
    asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float ieee_mul(float a, float b)
{
    float r;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float ieee_fma(float a, float b, float c)
{
    float r;
    asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
// The falloff G = e^q, q = -0.5 A' dx^2 - B' dx dy - 0.5 C' dy^2, is evaluated as 2^p with
// p = q log2 e: the per-entry factors (-A'/2, -B', -C'/2) are scaled by log2 e (rounded to
// FP32) once when the entry is staged, p is assembled per pixel from them, and 2^p is the
// hardware base-2 exponential (PTX ex2.approx, flush-to-zero: a result that would be denormal
// becomes zero, and o G is then below 1/255 either way).  p has the sign of q, so the
// "power > 0" guard reads p.
__device__ __forceinline__ float4 power_factors(const float4& conic)
{
    const float l2e = 1.44269502f;  // log2(e) rounded to FP32
    return make_float4(ieee_mul(ieee_mul(-0.5f, conic.x), l2e), ieee_mul(ieee_mul(-1.0f, conic.y), l2e),
                       ieee_mul(ieee_mul(-0.5f, conic.z), l2e), 0.0f);
}

__device__ __forceinline__ float gauss_exp2(float p)
{
    float g;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(p));
    return g;
}

// ---- a lane's two pixels as packed FP32 pairs --------------------------------------------
// A lane holds pixels (px, py0) and (px, py0 + 4), so every per-pixel quantity is a pair and
// one packed FP32x2 instruction updates both.  The pairs that decide skip and stop use explicit
// IEEE instructions (round to nearest, denormals kept), per component identical to the scalar
// ones, so both kernels compute the same bits.
__device__ __forceinline__ unsigned long long pk2(float2 v)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 ieee_sub2(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
__device__ __forceinline__ float2 ieee_mul2(float2 a, float2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
__device__ __forceinline__ float2 ieee_fma2(float2 a, float2 b, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
    return upk2(r);
}

// A staged entry of a tile's list, laid out so that the values a packed instruction needs on
// both pixels sit in aligned register pairs of one 16-byte shared-memory load:
//   e0 = (v, v, hC, hC)          v: screen y of the centre; hC = -C'/2 log2 e
//   e1 = (u, hA, hB, -o)         u: screen x; hA = -A'/2 log2 e, hB = -B' log2 e; -opacity
//   e2 = (-o, -o, r, r)
//   e3 = (g, g, b, b)            the view-dependent colour
// Opacity is staged negated: -alpha = max(-0.99, (-o) 2^p) is then exact, T (1 - alpha) is
// one fused multiply-add fma(-alpha, T, T), and no per-pair negation is needed.
struct Staged {
    float4 e0, e1, e2, e3;
};

__device__ __forceinline__ Staged stage_entry(const float4& a, const float4& conic, const float4& c)
{
    const float4 nf = power_factors(conic);
    Staged s;
    s.e0 = make_float4(a.y, a.y, nf.z, nf.z);
    s.e1 = make_float4(a.x, nf.x, nf.y, -a.z);
    s.e2 = make_float4(-a.z, -a.z, c.x, c.x);
    s.e3 = make_float4(c.y, c.y, c.z, c.z);
    return s;
}

// p = log2(e) times the power of Eq. 1 at both pixels of a lane from a staged entry, in the
// operations and order of the oracle's parity analysis: dx = u - px, dy = v - py,
// p = fma(hC dy, dy, fma(hB dx, dy, (hA dx) dx)).
__device__ __forceinline__ float2 staged_power2(const float4& e0, const float4& e1, float fpx, float2 fpy, float* dx_out,
                                                float2* dy_out)
{
    const float dx = ieee_sub(e1.x, fpx);
    const float ax = ieee_mul(ieee_mul(e1.y, dx), dx);
    const float nbx = ieee_mul(e1.z, dx);
    const float2 dy = ieee_sub2(make_float2(e0.x, e0.y), fpy);
    const float2 hcd = ieee_mul2(make_float2(e0.z, e0.w), dy);
    *dx_out = dx;
    *dy_out = dy;
    return ieee_fma2(hcd, dy, ieee_fma2(make_float2(nbx, nbx), dy, make_float2(ax, ax)));
}

// -alpha at both pixels: max(-0.99, (-o) 2^p), and (-o) 2^p itself (the clamp test reads it).
__device__ __forceinline__ float2 neg_alpha2(const float4& e2, float2 G, float2* nog)
{
    const float2 n = ieee_mul2(make_float2(e2.x, e2.y), G);
    *nog = n;
    return make_float2(fmaxf(-0.99f, n.x), fmaxf(-0.99f, n.y));
}

// ---- the parity build (cgs_config.exact) -------------------------------------------------
// The decisions of Eq. 1 in the operations and order of the plain per-pixel loop: with
// dx = u - px, dy = v - py, power = -0.5 ((A' dx) dx + (C' dy) dy) - (B' dx) dy, every
// operation rounded once; G = e^power rounded once to FP32 (the FP64 exponential, then one
// rounding); alpha = min(0.99, o G) (o G when o G < 0.99, else 0.99).  The transmittance then
// follows T (1 - alpha) and the colour C + c (alpha T), two roundings each.  One FP64
// exponential per pair: slow on this part, meant for parity checks.
__device__ __forceinline__ float exact_power(const float4& cn, float u, float v, float px, float py)
{
    const float dx = ieee_sub(u, px), dy = ieee_sub(v, py);
    const float s = ieee_add(ieee_mul(ieee_mul(cn.x, dx), dx), ieee_mul(ieee_mul(cn.z, dy), dy));
    return ieee_sub(ieee_mul(-0.5f, s), ieee_mul(ieee_mul(cn.y, dx), dy));
}

// o G with G = e^p rounded once to FP32.
__device__ __forceinline__ float exact_og(float o, float p)
{
    return ieee_mul(o, __double2float_rn(exp((double)p)));
}

__device__ __forceinline__ float exact_alpha(float og) { return og < 0.99f ? og : 0.99f; }

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

}  // namespace cgs
