// Shared pieces of the compositing kernels (stage d of the hot path: Eq. 1, Sec. 3.1, and its
// backward replay): the per-pair power, the per-warp culling masks, the forward blend and
// the backward replay of one pixel.
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

// p at a lane's two pixels (px, py0) and (px, py1), which share dx, from the entry's staged
// factors nf (power_factors).
__device__ __forceinline__ void pair_power2(const float4& a, const float4& nf, float fpx, float fpy0, float fpy1,
                                            float* pw0, float* pw1, float* dx_out, float* dy0_out, float* dy1_out)
{
    const float dx = ieee_sub(a.x, fpx), dy0 = ieee_sub(a.y, fpy0), dy1 = ieee_sub(a.y, fpy1);
    const float hC = nf.z;                               // -C'/2 log2 e
    const float ax = ieee_mul(ieee_mul(nf.x, dx), dx);   // -A' dx^2 / 2 log2 e
    const float nbx = ieee_mul(nf.y, dx);                // -B' dx log2 e
    *pw0 = ieee_fma(ieee_mul(hC, dy0), dy0, ieee_fma(nbx, dy0, ax));
    *pw1 = ieee_fma(ieee_mul(hC, dy1), dy1, ieee_fma(nbx, dy1, ax));
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
        const float alpha = fminf(0.99f, __fmul_rn(o, gauss_exp2(power)));
        const float Tn = ieee_fma(-alpha, T, T);  // T (1 - alpha), rounded once
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
        const float G = gauss_exp2(power);
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

}  // namespace cgs
