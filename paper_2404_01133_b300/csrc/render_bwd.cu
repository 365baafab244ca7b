// Backward of stage d (differentiable rendering, Sec. 3.1): every pixel replays its blended
// entries back to front from its final transmittance and n_contrib.  Built with
// flush-to-zero (denormal results of the gradient arithmetic become zero; the decisions that
// must match the forward are computed by render_common.cuh's explicit IEEE instructions or
// do not depend on denormals: a denormal exp() or opacity product is below 1/255 either way).
#include "render_common.cuh"

namespace cgs {

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
    __shared__ float4 s_a[BATCH], s_b[BATCH], s_c[BATCH], s_f[BATCH];
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
            const float4 cb = L.rec[3 * (size_t)j + 1];
            s_b[i] = cb;
            s_f[i] = power_factors(cb);
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
                    const float4 a = s_a[k], nf = s_f[k], c = s_c[k];
                    const uint32_t lp = (uint32_t)(bs + k - first);
                    float pw0, pw1, dx, dy0, dy1;
                    pair_power2(a, nf, fpx, fpy0, fpy1, &pw0, &pw1, &dx, &dy0, &dy1);
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
static void bwd_launch(const Layout& L, const uint32_t* tval, const cgs_config& c, const float* dimg, const float* T,
                       const uint32_t* nc, cudaStream_t st)
{
    dim3 grid(L.tiles_x, L.tiles_y, L.V);
    k_render_bwd<B, BATCH><<<grid, B * B / 2, 0, st>>>(L, tval, c.bg[0], c.bg[1], c.bg[2], dimg, T, nc);
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

}  // namespace cgs
