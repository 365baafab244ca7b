// Issue-rate peaks of the device, measured: the denominators of the compositing kernels'
// roofline (FP32 instructions and SFU exponentials per second).  Instrumentation only: the
// paper has no counterpart.
//
// Every loop keeps CHAINS independent dependency chains per thread so that latency is hidden,
// and runs on n_sm x 8 CTAs of 256 threads (64 resident warps per SM).  The kernels write one
// value per thread so that nothing is optimised away.
#include "common.cuh"

namespace cgs {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

// Scalar FP32 fused multiply-adds: PK_CHAINS per iteration.
__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(float* out, int iters, float a, float b)
{
    float x[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
#pragma unroll
            for (int k = 0; k < PK_CHAINS; k++) x[k] = __fmaf_rn(x[k], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed FP32 fused multiply-adds (two lanes' worth of work per instruction).
__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma2(float* out, int iters, float a, float b)
{
    float2 x[PK_CHAINS];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
#pragma unroll
            for (int k = 0; k < PK_CHAINS; k++) x[k] = __ffma2_rn(x[k], a2, b2);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) s += x[k].x + x[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Base-2 exponentials (the compositing kernels' one transcendental per pair): x <- 2^-x,
// which stays in [0.5, 1].
__global__ void __launch_bounds__(PK_THREADS) k_peak_ex2(float* out, int iters)
{
    float x[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) x[k] = 0.5f + (float)k * 0.01f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
#pragma unroll
            for (int k = 0; k < PK_CHAINS; k++) {
                float y;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[k]));
                x[k] = y;
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace cgs

using namespace cgs;

extern "C" int32_t cgs_measure_peaks(double* rates, int32_t n_rates, float* d_scratch, int64_t scratch_floats,
                                     void* stream)
{
    const int n_sm = device_sm_count();
    const int grid = n_sm * 8;
    if (!rates || n_rates < 3 || !d_scratch || scratch_floats < (int64_t)grid * PK_THREADS)
        return CGS_ERR_INVALID_ARGUMENT;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CGS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CGS_ERR_CUDA;
    }
    const int iters = 4096;
    const double threads = (double)grid * PK_THREADS;
    // lane operations per launch: iterations x 4 unrolled x chains (x2 for the packed form)
    const double ops[3] = {threads * iters * 4.0 * PK_CHAINS, threads * iters * 4.0 * PK_CHAINS * 2.0,
                           threads * iters * 4.0 * PK_CHAINS};
    int32_t rc = CGS_OK;
    for (int which = 0; which < 3 && rc == CGS_OK; which++) {
        float best = 0.0f;
        for (int rep = 0; rep < 4; rep++) {  // the first launch warms up; best of the others
            cudaEventRecord(e0, st);
            if (which == 0) k_peak_ffma<<<grid, PK_THREADS, 0, st>>>(d_scratch, iters, 0.999f, 1e-3f);
            else if (which == 1) k_peak_ffma2<<<grid, PK_THREADS, 0, st>>>(d_scratch, iters, 0.999f, 1e-3f);
            else k_peak_ex2<<<grid, PK_THREADS, 0, st>>>(d_scratch, iters);
            cudaEventRecord(e1, st);
            count_launches(1);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = CGS_ERR_CUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
        }
        if (rc == CGS_OK) rates[which] = best > 0.0f ? ops[which] / (best * 1e-3) : 0.0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) rc = CGS_ERR_CUDA;
    return rc;
}
