// Detail levels of a block-grouped scene (Sec. 3.3.1): inside every block, rank the Gaussians
// by a significance score and keep nested prefixes of that order as the levels.
//
//   score    o * ((s_x * s_y) * s_z), times (float)h when per-Gaussian hit counts h are given
//            (pixels whose compositing blends the Gaussian, counted by the forward render);
//            FP32 in this order, NaN ranked as -inf
//   order    per block: descending score, equal scores by increasing row
//   levels   level l of a block of K rows keeps its first floor(K rate_l) rows (FP64 product)
//
// The order is one stable LSD radix sort of 64-bit keys (block << 32 | descending score key),
// eight bits per pass, rows as values: the low four passes order by score, the high passes
// (one per eight bits of the block count) restore the block grouping; stability gives equal
// scores in row order.  Every pass is a counting sort over warp-owned chunks: a per-chunk
// digit histogram in warp-private shared memory, a single-pass scan in (digit, chunk) order,
// and a stable scatter that ranks equal digits inside a warp with eight ballots.  Both
// kernels load several 32-key groups before using any, to keep enough bytes in flight.
#include <algorithm>
#include <cmath>

#include <cuda_fp16.h>

#include "common.cuh"
#include "scan.cuh"

namespace cgs {

constexpr int RX_WARPS = 8;
constexpr int RX_THREADS = 32 * RX_WARPS;
constexpr int RX_BUCKETS = 256;
constexpr int RX_MIN_CHUNK = 1024;
constexpr long long RX_MAX_COUNTS = 1ll << 23;
constexpr int RX_MAX_PASSES = 6;  // 4 score passes + up to 2 block passes (1024 blocks)
constexpr int RX_ILP = 8;         // groups of 32 keys loaded before any is ranked

struct LevelRates {
    double r[CGS_MAX_LEVELS];
};

__device__ __forceinline__ float half_bits_to_float(unsigned short b) { return __half2float(__ushort_as_half(b)); }

// Descending-order key of a score: larger scores give smaller keys; NaN ranks as -inf and
// -0 with +0 (both decided on the bit pattern).
__device__ __forceinline__ uint32_t desc_key(float s)
{
    uint32_t u = __float_as_uint(s);
    if ((u & 0x7fffffffu) > 0x7f800000u) u = 0xff800000u;  // NaN -> -inf
    if ((u & 0x7fffffffu) == 0u) u = 0u;                   // -0 -> +0
    const uint32_t asc = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ~asc;
}

__global__ void __launch_bounds__(256) k_level_keys(const float* __restrict__ mo, const void* __restrict__ scale,
                                                    int fp16, const uint32_t* __restrict__ hits,
                                                    const int64_t* __restrict__ off, int nb, long long n,
                                                    unsigned long long* __restrict__ keys, int32_t* __restrict__ vals)
{
    __shared__ long long s_off[CGS_PARTITION_MAX_BLOCKS + 1];
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) s_off[b] = off[b];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        // block: the largest b < nb with off[b] <= i
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        float s0, s1, s2;
        if (fp16) {
            const uint2 a = __ldg(reinterpret_cast<const uint2*>(scale) + i);
            s0 = half_bits_to_float(a.x & 0xffffu);
            s1 = half_bits_to_float(a.x >> 16);
            s2 = half_bits_to_float(a.y & 0xffffu);
        } else {
            const float4 a = __ldg(reinterpret_cast<const float4*>(scale) + i);
            s0 = a.x; s1 = a.y; s2 = a.z;
        }
        const float o = __ldg(mo + 4 * i + 3);
        const float vol = __fmul_rn(__fmul_rn(s0, s1), s2);
        float sc = __fmul_rn(o, vol);
        if (hits) sc = __fmul_rn(__uint2float_rn(__ldg(hits + i)), sc);
        keys[i] = ((unsigned long long)lo << 32) | desc_key(sc);
        vals[i] = (int32_t)i;
    }
}

__global__ void __launch_bounds__(256) k_level_counts(const int64_t* __restrict__ off, int nb, LevelRates R, int nl,
                                                      int64_t* __restrict__ level_count)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * nl) return;
    const int b = t / nl, l = t - b * nl;
    const long long K = off[b + 1] - off[b];
    level_count[t] = (int64_t)floor(__dmul_rn((double)K, R.r[l]));
}

// Digit histogram of every chunk.  A warp walks its chunk RX_ILP groups of 32 keys at a time,
// with all the group loads issued before any is counted (memory parallelism); counts go to
// warp-private shared-memory counters (the order of the additions does not matter).
__global__ void __launch_bounds__(RX_THREADS) k_radix_hist(const unsigned long long* __restrict__ keys, long long n,
                                                           int shift, long long ch, long long n_chunks,
                                                           uint32_t* __restrict__ cnt)
{
    __shared__ uint32_t s_hist[RX_WARPS][RX_BUCKETS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* hist = s_hist[warp];
    for (int b = lane; b < RX_BUCKETS; b += 32) hist[b] = 0;
    __syncwarp();
    const long long gw = (long long)blockIdx.x * RX_WARPS + warp, nw = (long long)gridDim.x * RX_WARPS;
    for (long long chunk = gw; chunk < n_chunks; chunk += nw) {
        const long long c0 = chunk * ch, c1 = min(n, c0 + ch);
        for (long long base = c0; base < c1; base += 32 * RX_ILP) {
            unsigned long long k[RX_ILP];
#pragma unroll
            for (int u = 0; u < RX_ILP; u++) {
                const long long i = base + u * 32 + lane;
                k[u] = i < c1 ? __ldg(keys + i) : ~0ull;
            }
#pragma unroll
            for (int u = 0; u < RX_ILP; u++)
                if (base + u * 32 + lane < c1) atomicAdd(&hist[(k[u] >> shift) & 0xffu], 1u);
        }
        __syncwarp();
        for (int b = lane; b < RX_BUCKETS; b += 32) {
            cnt[(long long)b * n_chunks + chunk] = hist[b];
            hist[b] = 0;
        }
        __syncwarp();
    }
}

struct RadixScanOp {
    uint32_t* cnt;
    long long total;
    __device__ long long count() const { return total; }
    __device__ uint32_t load(long long t) const { return cnt[t]; }
    __device__ void store(long long t, unsigned long long e, uint32_t x) const
    {
        (void)x;
        cnt[t] = (uint32_t)e;
    }
    __device__ void finish(unsigned long long tot) const { (void)tot; }
};

// Lanes of the warp holding the same 8-bit digit d (among the lanes in `valid`): eight ballots.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, uint32_t valid)
{
    uint32_t peers = valid;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const uint32_t m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? m : ~m;
    }
    return peers;
}

// Stable scatter of one pass.  The warp loads RX_ILP groups of its chunk up front, then ranks
// them group by group in chunk order: slot = the chunk's running count of the digit + the
// number of earlier lanes of the group with the same digit.
__global__ void __launch_bounds__(RX_THREADS) k_radix_scatter(const unsigned long long* __restrict__ kin,
                                                              const int32_t* __restrict__ vin,
                                                              unsigned long long* __restrict__ kout,
                                                              int32_t* __restrict__ vout, long long n, int shift,
                                                              long long ch, long long n_chunks,
                                                              const uint32_t* __restrict__ base)
{
    __shared__ uint32_t s_run[RX_WARPS][RX_BUCKETS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* run = s_run[warp];
    const uint32_t lt = (1u << lane) - 1u;
    const long long gw = (long long)blockIdx.x * RX_WARPS + warp, nw = (long long)gridDim.x * RX_WARPS;
    for (long long chunk = gw; chunk < n_chunks; chunk += nw) {
        for (int b = lane; b < RX_BUCKETS; b += 32) run[b] = __ldg(base + (long long)b * n_chunks + chunk);
        __syncwarp();
        const long long c0 = chunk * ch, c1 = min(n, c0 + ch);
        for (long long b0 = c0; b0 < c1; b0 += 32 * RX_ILP) {
            unsigned long long k[RX_ILP];
            int32_t v[RX_ILP];
#pragma unroll
            for (int u = 0; u < RX_ILP; u++) {
                const long long i = b0 + u * 32 + lane;
                k[u] = 0;
                v[u] = 0;
                if (i < c1) {
                    k[u] = __ldg(kin + i);
                    v[u] = __ldg(vin + i);
                }
            }
#pragma unroll
            for (int u = 0; u < RX_ILP; u++) {
                const bool ok = b0 + u * 32 + lane < c1;
                const uint32_t valid = __ballot_sync(0xffffffffu, ok);
                if (!valid) break;
                const uint32_t d = (uint32_t)(k[u] >> shift) & 0xffu;
                const uint32_t peers = digit_peers(d, valid);
                uint32_t slot = 0;
                if (ok) slot = run[d] + __popc(peers & lt);
                __syncwarp();
                if (ok) {
                    if (kout) kout[slot] = k[u];
                    vout[slot] = v[u];
                    if (lane == __ffs(peers) - 1) run[d] += __popc(peers);
                }
                __syncwarp();
            }
        }
    }
}

struct RxPlan {
    long long ch, n_chunks, counts;
    int passes;
    size_t off_keys0, off_keys1, off_vals0, off_vals1, off_cnt, off_lb, lb_bytes, total;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static RxPlan rx_plan(long long n, int nb)
{
    RxPlan p;
    long long ch = (n * RX_BUCKETS + RX_MAX_COUNTS - 1) / RX_MAX_COUNTS;
    ch = ((ch + 31) / 32) * 32;
    p.ch = ch < RX_MIN_CHUNK ? RX_MIN_CHUNK : ch;
    p.n_chunks = n > 0 ? (n + p.ch - 1) / p.ch : 1;
    p.counts = p.n_chunks * RX_BUCKETS;
    int hi_bits = 0;
    while ((1ll << hi_bits) < nb) hi_bits++;
    p.passes = 4 + (hi_bits + 7) / 8;
    size_t o = al256(sizeof(Header));
    p.off_keys0 = o; o = al256(o + (size_t)n * 8);
    p.off_keys1 = o; o = al256(o + (size_t)n * 8);
    p.off_vals0 = o; o = al256(o + (size_t)n * 4);
    p.off_vals1 = o; o = al256(o + (size_t)n * 4);
    p.off_cnt = o; o = al256(o + (size_t)p.counts * 4);
    p.lb_bytes = al256((size_t)((p.counts + SCAN_TILE - 1) / SCAN_TILE) * 8);
    p.off_lb = o; o += p.lb_bytes * RX_MAX_PASSES;
    p.total = o;
    return p;
}

}  // namespace cgs

using namespace cgs;

extern "C" int64_t cgs_levels_workspace_bytes(int64_t n, int32_t n_blocks)
{
    if (n < 0 || n >= (1ll << 31) || n_blocks < 1 || n_blocks > CGS_PARTITION_MAX_BLOCKS) return -1;
    return (int64_t)rx_plan(n, n_blocks).total;
}

extern "C" int32_t cgs_generate_levels(const float* d_mean_opac, const void* d_scale, int32_t attr_fp16, int64_t n,
                                       const int64_t* d_block_offset, int32_t n_blocks, const uint32_t* d_hits,
                                       const double* rates, int32_t n_levels, int32_t* d_perm,
                                       int64_t* d_level_count, void* d_ws, int64_t ws_bytes, void* stream)
{
    if (n < 0 || n >= (1ll << 31) || n_blocks < 1 || n_blocks > CGS_PARTITION_MAX_BLOCKS || !d_block_offset ||
        !rates || n_levels < 1 || n_levels > CGS_MAX_LEVELS || !d_level_count || (attr_fp16 != 0 && attr_fp16 != 1))
        return CGS_ERR_INVALID_ARGUMENT;
    if (n > 0 && (!d_mean_opac || !d_scale || !d_perm)) return CGS_ERR_INVALID_ARGUMENT;
    LevelRates R;
    for (int l = 0; l < CGS_MAX_LEVELS; l++) R.r[l] = 0.0;
    for (int l = 0; l < n_levels; l++) {
        if (!(rates[l] >= 0.0 && rates[l] <= 1.0)) return CGS_ERR_INVALID_ARGUMENT;
        R.r[l] = rates[l];
    }
    const RxPlan p = rx_plan(n, n_blocks);
    if (!d_ws || ws_bytes < (int64_t)p.total) return CGS_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = static_cast<char*>(d_ws);
    Header* hdr = reinterpret_cast<Header*>(ws);
    unsigned long long* keys[2] = {reinterpret_cast<unsigned long long*>(ws + p.off_keys0),
                                   reinterpret_cast<unsigned long long*>(ws + p.off_keys1)};
    int32_t* vals[2] = {reinterpret_cast<int32_t*>(ws + p.off_vals0), reinterpret_cast<int32_t*>(ws + p.off_vals1)};
    uint32_t* cnt = reinterpret_cast<uint32_t*>(ws + p.off_cnt);
    char* lb = ws + p.off_lb;
    if (cudaMemsetAsync(hdr, 0, sizeof(Header), st) != cudaSuccess) return CGS_ERR_CUDA;
    if (cudaMemsetAsync(lb, 0, p.lb_bytes * RX_MAX_PASSES, st) != cudaSuccess) return CGS_ERR_CUDA;
    const int n_sm = device_sm_count();
    int launched = 0;
    {
        const int t = n_blocks * n_levels;
        k_level_counts<<<(t + 255) / 256, 256, 0, st>>>(d_block_offset, n_blocks, R, n_levels, d_level_count);
        launched++;
    }
    if (n > 0) {
        const long long g = std::min<long long>((n + 255) / 256, (long long)n_sm * 8);
        k_level_keys<<<(unsigned)g, 256, 0, st>>>(d_mean_opac, d_scale, attr_fp16, d_hits, d_block_offset, n_blocks, n,
                                                  keys[0], vals[0]);
        launched++;
        const long long ctas = std::max<long long>(
            1, std::min<long long>((p.n_chunks + RX_WARPS - 1) / RX_WARPS, (long long)n_sm * 4));
        const long long scan_ctas = std::max<long long>(
            1, std::min<long long>((p.counts + SCAN_TILE - 1) / SCAN_TILE, (long long)n_sm * 8));
        int cur = 0;
        for (int pass = 0; pass < p.passes; pass++) {
            const int shift = 8 * pass;
            const bool last = pass == p.passes - 1;
            k_radix_hist<<<(unsigned)ctas, RX_THREADS, 0, st>>>(keys[cur], n, shift, p.ch, p.n_chunks, cnt);
            RadixScanOp op{cnt, p.counts};
            k_scan<RadixScanOp><<<(unsigned)scan_ctas, SCAN_THREADS, 0, st>>>(
                op, reinterpret_cast<unsigned long long*>(lb + p.lb_bytes * pass), hdr->ctr + pass, hdr);
            k_radix_scatter<<<(unsigned)ctas, RX_THREADS, 0, st>>>(keys[cur], vals[cur], last ? nullptr : keys[cur ^ 1],
                                                                   last ? d_perm : vals[cur ^ 1], n, shift, p.ch,
                                                                   p.n_chunks, cnt);
            launched += 3;
            cur ^= 1;
        }
    }
    count_launches(launched);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

extern "C" int32_t cgs_levels_status(const void* d_ws, void* stream)
{
    if (!d_ws) return CGS_ERR_INVALID_ARGUMENT;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CGS_ERR_CUDA;
    Header h;
    if (cudaMemcpy(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return CGS_ERR_CUDA;
    return (h.status & ST_SPIN) ? CGS_ERR_SPIN_TIMEOUT : CGS_OK;
}
