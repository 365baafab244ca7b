// Structural similarity of renders, for the SSIM loss of Eq. 3 (B1 pose assignment,
// Sec. 3.2.2): per channel, local means, variances and covariance under an 11 x 11 Gaussian
// window (sigma 1.5, weights summing to 1, zero outside the image), the SSIM map
//   ((2 mu_a mu_b + C1)(2 s_ab + C2)) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 + s_b^2 + C2)),
// C1 = 0.01^2, C2 = 0.03^2, averaged over every pixel and channel.
//
// One CTA per 32 x 16 output tile of one image pair: the 42 x 26 input window of both images
// is staged in shared memory per channel, the five products are filtered horizontally into
// shared memory and then vertically (the window is separable), and the CTA's sum of the map
// is added to the pair's mean with one atomic add.
#include <cmath>

#include "common.cuh"

namespace cgs {

constexpr int SS_TX = 32, SS_TY = 16, SS_R = 5;
constexpr int SS_IX = SS_TX + 2 * SS_R, SS_IY = SS_TY + 2 * SS_R;
constexpr int SS_THREADS = 256;

struct SsimWindow {
    float g[2 * SS_R + 1];
};

__global__ void __launch_bounds__(SS_THREADS) k_ssim(const float* __restrict__ a, long long a_stride,
                                                     const float* __restrict__ b, int C, int W, int H, SsimWindow wnd,
                                                     float inv_count, float* __restrict__ out, float* __restrict__ map)
{
    __shared__ float s_a[SS_IY][SS_IX], s_b[SS_IY][SS_IX];
    __shared__ float s_h[5][SS_IY][SS_TX];
    __shared__ float s_sum[SS_THREADS / 32];
    const int pair = blockIdx.z;
    const int x0 = blockIdx.x * SS_TX, y0 = blockIdx.y * SS_TY;
    const long long plane = (long long)W * H;
    const float* A = a + (long long)pair * a_stride;
    const float* B = b + (long long)pair * C * plane;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float acc = 0.0f;
    // each thread owns two output pixels of the tile: (tx, ty) and (tx, ty + 8)
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float msum[2] = {0.0f, 0.0f};
    for (int c = 0; c < C; c++) {
        __syncthreads();
        for (int i = threadIdx.x; i < SS_IX * SS_IY; i += SS_THREADS) {
            const int iy = i / SS_IX, ix = i - iy * SS_IX;
            const int gx = x0 + ix - SS_R, gy = y0 + iy - SS_R;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            s_a[iy][ix] = in ? __ldg(A + c * plane + (long long)gy * W + gx) : 0.0f;
            s_b[iy][ix] = in ? __ldg(B + c * plane + (long long)gy * W + gx) : 0.0f;
        }
        __syncthreads();
        // horizontal pass over every staged row
        for (int i = threadIdx.x; i < SS_IY * SS_TX; i += SS_THREADS) {
            const int iy = i / SS_TX, ox = i - iy * SS_TX;
            float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
            for (int k = 0; k < 2 * SS_R + 1; k++) {
                const float va = s_a[iy][ox + k], vb = s_b[iy][ox + k], w = wnd.g[k];
                m0 += w * va;
                m1 += w * vb;
                m2 += w * va * va;
                m3 += w * vb * vb;
                m4 += w * va * vb;
            }
            s_h[0][iy][ox] = m0;
            s_h[1][iy][ox] = m1;
            s_h[2][iy][ox] = m2;
            s_h[3][iy][ox] = m3;
            s_h[4][iy][ox] = m4;
        }
        __syncthreads();
        // vertical pass and the map
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int oy = ty + 8 * h;
            float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 2 * SS_R + 1; k++) {
                const float w = wnd.g[k];
#pragma unroll
                for (int q = 0; q < 5; q++) m[q] += w * s_h[q][oy + k][tx];
            }
            const float ma = m[0], mb = m[1];
            const float va = m[2] - ma * ma, vb = m[3] - mb * mb, cv = m[4] - ma * mb;
            const float v = ((2.0f * ma * mb + C1) * (2.0f * cv + C2)) / ((ma * ma + mb * mb + C1) * (va + vb + C2));
            if (x0 + tx < W && y0 + oy < H) {
                acc += v;
                msum[h] += v;
            }
        }
    }
    if (map) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int gx = x0 + tx, gy = y0 + ty + 8 * h;
            if (gx < W && gy < H) map[(long long)pair * plane + (long long)gy * W + gx] = msum[h] / (float)C;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < SS_THREADS / 32; w++) t += s_sum[w];
        atomicAdd(out + pair, t * inv_count);
    }
}

}  // namespace cgs

using namespace cgs;

extern "C" int32_t cgs_ssim(const float* d_a, int64_t a_stride, const float* d_b, int32_t n_pairs, int32_t channels,
                            int32_t width, int32_t height, float* d_ssim, float* d_map, void* stream)
{
    if (!d_a || !d_b || !d_ssim || n_pairs < 1 || n_pairs > 65535 || channels < 1 || width < 1 || height < 1 ||
        a_stride < 0)
        return CGS_ERR_INVALID_ARGUMENT;
    SsimWindow wnd;
    double g[2 * SS_R + 1], s = 0.0;
    for (int k = 0; k <= 2 * SS_R; k++) {
        const double d = (double)(k - SS_R);
        g[k] = std::exp(-(d * d) / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    for (int k = 0; k <= 2 * SS_R; k++) wnd.g[k] = (float)(g[k] / s);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(d_ssim, 0, sizeof(float) * (size_t)n_pairs, st) != cudaSuccess) return CGS_ERR_CUDA;
    dim3 grid((width + SS_TX - 1) / SS_TX, (height + SS_TY - 1) / SS_TY, n_pairs);
    const float inv = (float)(1.0 / ((double)channels * (double)width * (double)height));
    k_ssim<<<grid, SS_THREADS, 0, st>>>(d_a, a_stride, d_b, channels, width, height, wnd, inv, d_ssim, d_map);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}
