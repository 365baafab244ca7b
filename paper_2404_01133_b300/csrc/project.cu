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
// by that slack, the extent is infinite (never culled).  Opacity below 1/255 can never pass
// the test: extent -1 (always culled).
// *tq receives the slackened threshold t itself (for the exact ellipse test of the
// compositing kernels), or +inf when no culling is safe.
__device__ __forceinline__ void cull_extent(float o, float A, float B, float C, float* ex, float* ey, float* tq)
{
    if (!(o * 255.0f > 1.0f)) { *ex = -1.0f; *ey = -1.0f; *tq = -1.0f; return; }
    if (B * B > 0.99f * A * C) { *ex = INFINITY; *ey = INFINITY; *tq = INFINITY; return; }
    const float t = 2.0f * logf(255.0f * o) * 1.002f + 0.002f;
    *ex = sqrtf(t * A) * 1.001f + 0.01f;
    *ey = sqrtf(t * C) * 1.001f + 0.01f;
    *tq = t;
}

// One thread per selected Gaussian j (flattened over views), grid-stride over the device
// count written by the selection kernels.  Writes tiles touched and the scene index of every
// selected Gaussian and, for the visible ones, the screen-space part of the projected record,
// the tile rect, the (view, depth) sort key and cleared screen-gradient accumulators.  Colour
// is evaluated later by k_colour over the compacted visible list.
__global__ void __launch_bounds__(256) k_project(Layout L, cgs_scene S, const cgs_camera* __restrict__ cams,
                                                 float near_z)
{
    const uint32_t n = L.hdr->n_sel;
    const float4* __restrict__ mo4 = reinterpret_cast<const float4*>(S.mean_opac);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int v;
        long long g;
        locate(L, j, &v, &g);
        L.gidx[j] = (uint32_t)g;
        const cgs_camera& c = cams[v];
        const float4 mo = __ldg(mo4 + g);
        const float m[3] = {mo.x, mo.y, mo.z};
        // near-plane test first, so culled Gaussians never read scale or rotation
        const float tz = ((c.R[6] * m[0] + c.R[7] * m[1]) + c.R[8] * m[2]) + c.t[2];
        uint32_t tt = 0;
        bool keep = tz > near_z;
        if (keep && L.lod_mode == CGS_LOD_POINT) {
            // point-wise baseline: the level of this Gaussian's own distance; kept iff its rank
            // in the block lies inside that level's (nested) prefix
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
                    L.rect[j] = make_uint2(tx0 | (ty0 << 16), tx1 | (ty1 << 16));
                    float ex, ey, tq;
                    cull_extent(mo.w, p.A, p.B, p.C, &ex, &ey, &tq);
                    L.tq[j] = tq;
                    L.rec[3 * (size_t)j] = make_float4(p.u, p.v, mo.w, ex);
                    L.rec[3 * (size_t)j + 1] = make_float4(p.conic[0], p.conic[1], p.conic[2], ey);
                    L.pkey[j] = ((unsigned long long)(uint32_t)v << 32) | __float_as_uint(p.tz);
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    L.gs[3 * (size_t)j] = z4;
                    L.gs[3 * (size_t)j + 1] = z4;
                    L.gs[3 * (size_t)j + 2] = z4;
                }
            }
        }
        L.tt[j] = tt;
    }
}

// View-dependent colour (SH, Sec. 3.1) of each visible Gaussian, over the compacted visible
// list so every lane has work.  Writes the third record (r, g, b, t), t the culling
// threshold on the quadratic form (see cull_extent).
__global__ void __launch_bounds__(256) k_colour(Layout L, cgs_scene S, const cgs_camera* __restrict__ cams)
{
    const uint32_t n = L.hdr->n_vis;
    const int deg = S.sh_degree;
    const int nc = (deg + 1) * (deg + 1);
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const uint32_t j = L.vis[r];
        const int v = (int)(L.pkey[j] >> 32);
        const long long g = L.gidx[j];
        const float4 mo = __ldg(reinterpret_cast<const float4*>(S.mean_opac) + g);
        const float m[3] = {mo.x, mo.y, mo.z};
        float f[48], rgb[3], dir[3], len, Y[16];
        if (S.attr_fp16) load_sh_half(S.sh, g, nc, f);
        else load_sh(S.sh, g, nc, f);
        sh_colour(m, cams[v], f, deg, rgb, dir, &len, Y);
        L.rec[3 * (size_t)j + 2] = make_float4(rgb[0], rgb[1], rgb[2], L.tq[j]);
    }
}

void launch_project(const Layout& L, const cgs_scene& S, const cgs_camera* cams, float near_z, int n_sm,
                    cudaStream_t st)
{
    long long want = (L.n_cap + 255) / 256;
    long long grid = want < (long long)n_sm * 8 ? want : (long long)n_sm * 8;
    if (grid < 1) grid = 1;
    k_project<<<(unsigned)grid, 256, 0, st>>>(L, S, cams, near_z);
}

void launch_colour(const Layout& L, const cgs_scene& S, const cgs_camera* cams, int n_sm, cudaStream_t st)
{
    long long want = (L.n_cap + 255) / 256;
    long long grid = want < (long long)n_sm * 8 ? want : (long long)n_sm * 8;
    if (grid < 1) grid = 1;
    k_colour<<<(unsigned)grid, 256, 0, st>>>(L, S, cams);
}

}  // namespace cgs
