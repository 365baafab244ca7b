// Stage c of the hot path, after the projection has emitted the (tile, Gaussian) entries and
// the per-tile counts: the depth order inside every tile ("sorted in depth order", Sec. 3.1;
// ties to the lower index).
//
//   tile ranges   single-pass scan of the per-tile counts -> [start, end) of every tile
//   scatter       one thread per entry: a slot in its tile's range (atomic cursor), key
//                 (FP32 depth bits << 32 | selected index)
//   tile sort     one CTA per tile: up to 256 keys ranked against each other in shared
//                 memory (each key's count of smaller keys is its slot), up to 2048 keys
//                 bitonic-sorted in shared memory; longer tiles are sorted by one CTA of a
//                 second kernel (bitonic in shared memory up to 4096 keys, beyond that
//                 sorted chunks + merge rounds through global scratch)
//
// Within a view, a Gaussian appears at most once per tile, so the 64-bit keys of one tile are
// distinct: the sorted order is exactly (depth, index) whatever order the projection emitted
// the entries in and the scatter placed them.  Every count the sequence needs is read on the
// device; every inter-block wait is bounded and latches ST_SPIN.
#include "common.cuh"
#include "scan.cuh"

namespace cgs {

// [start, end) of every (view, tile) from the per-tile counts.
struct TileRangeOp {
    Layout L;
    __device__ long long count() const { return (long long)L.V * L.T; }
    __device__ uint32_t load(long long t) const { return L.tcnt[t]; }
    __device__ void store(long long t, unsigned long long e, uint32_t x) const
    {
        L.ranges[2 * t] = (uint32_t)e;
        L.ranges[2 * t + 1] = (uint32_t)(e + x);
    }
    __device__ void finish(unsigned long long total) const { (void)total; }
};

// One thread per entry: a slot inside its tile's range and the (depth bits, index) key.
__global__ void __launch_bounds__(256) k_scatter(Layout L)
{
    const long long n = entries_kept(L);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const unsigned long long w = L.eraw[k];
        const uint32_t t = (uint32_t)(w >> 32), j = (uint32_t)w;
        const uint32_t slot = L.ranges[2 * (size_t)t] + atomicAdd(&L.tcur[t], 1u);
        L.ekey[slot] = ((unsigned long long)(uint32_t)L.pkey[j] << 32) | j;
    }
}

constexpr int TS_THREADS = 256;
constexpr int TS_CAP = 2048;  // keys per tile sorted entirely in shared memory by k_tile_sort
constexpr int LT_CAP = 4096;  // keys per chunk of the long-tile kernel

// In-place ascending bitonic sort of s[0, np) (np a power of two) by the threads of a CTA.
__device__ __forceinline__ void bitonic_smem(unsigned long long* s, int np)
{
    for (int size = 2; size <= np; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (np >> 1); i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = s[lo], b = s[hi];
                if ((a > b) == up) { s[lo] = b; s[hi] = a; }
            }
        }
    }
    __syncthreads();
}

constexpr int RANK_MAX = TS_THREADS;  // keys per tile sorted by ranking

// One CTA per (view, tile).  Up to RANK_MAX keys: every thread ranks one key against all keys
// of the tile in shared memory (keys are distinct, so the rank is the output slot); up to
// TS_CAP keys: bitonic sort in shared memory; longer tiles are listed for the long-tile
// kernel.
__global__ void __launch_bounds__(TS_THREADS) k_tile_sort(Layout L)
{
    __shared__ unsigned long long s[TS_CAP];
    const uint32_t t = blockIdx.x;
    const uint32_t st = L.ranges[2 * (size_t)t], n = L.ranges[2 * (size_t)t + 1] - st;
    if (n == 0) return;
    if (n > (uint32_t)TS_CAP) {
        if (threadIdx.x == 0) L.big[atomicAdd(&L.hdr->n_big, 1u)] = t;
        return;
    }
    if (n <= (uint32_t)RANK_MAX) {
        const uint32_t i = threadIdx.x;
        const unsigned long long key = i < n ? L.ekey[st + i] : ~0ull;
        if (i < n) s[i] = key;
        __syncthreads();
        if (i < n) {
            uint32_t r = 0;
#pragma unroll 4
            for (uint32_t m = 0; m < n; m++) r += s[m] < key;
            L.tval[st + r] = (uint32_t)key;
            L.tkey[st + r] = t;
        }
        return;
    }
    int np = 2;
    while (np < (int)n) np <<= 1;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s[i] = i < (int)n ? L.ekey[st + i] : ~0ull;
    bitonic_smem(s, np);
    for (int i = threadIdx.x; i < (int)n; i += blockDim.x) {
        L.tval[st + i] = (uint32_t)s[i];
        L.tkey[st + i] = t;
    }
}

// Tiles longer than TS_CAP: one CTA per tile (persistent over the device list) sorts chunks
// of LT_CAP keys in shared memory (the whole tile when it fits), then merges runs pairwise
// through global scratch (the entry buffer, free after the scatter).  With distinct keys, an
// element's output position is its rank in its own run plus the number of smaller keys in
// the other run.
constexpr int TB_THREADS = 512;
__global__ void __launch_bounds__(TB_THREADS) k_tile_sort_large(Layout L)
{
    __shared__ unsigned long long s[LT_CAP];
    __shared__ uint32_t s_item;
    const uint32_t nbig = L.hdr->n_big;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&L.hdr->ctr[CTR_BIG], 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= nbig) break;
        const uint32_t t = L.big[item];
        const uint32_t st = L.ranges[2 * (size_t)t], n = L.ranges[2 * (size_t)t + 1] - st;
        unsigned long long* a = L.ekey + st;
        unsigned long long* b = L.eraw + st;
        for (uint32_t c0 = 0; c0 < n; c0 += LT_CAP) {
            const int m = (int)min((uint32_t)LT_CAP, n - c0);
            int np = 2;
            while (np < m) np <<= 1;
            for (int i = threadIdx.x; i < np; i += blockDim.x) s[i] = i < m ? a[c0 + i] : ~0ull;
            bitonic_smem(s, np);
            for (int i = threadIdx.x; i < m; i += blockDim.x) a[c0 + i] = s[i];
            __syncthreads();
        }
        for (uint32_t width = LT_CAP; width < n; width <<= 1) {
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                const uint32_t base = i - i % (2 * width);
                const bool in_first = (i - base) < width;
                const uint32_t a0 = base, a1 = min(base + width, n), b0 = a1, b1 = min(base + 2 * width, n);
                const unsigned long long key = a[i];
                uint32_t lo = in_first ? b0 : a0, hi = in_first ? b1 : a1;  // count keys < key in the other run
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (a[mid] < key) lo = mid + 1; else hi = mid;
                }
                const uint32_t other = lo - (in_first ? b0 : a0);
                const uint32_t own = i - (in_first ? a0 : b0);
                b[base + own + other] = key;
            }
            __syncthreads();
            unsigned long long* tmp = a;
            a = b;
            b = tmp;
        }
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            L.tval[st + i] = (uint32_t)a[i];
            L.tkey[st + i] = t;
        }
        __syncthreads();
    }
}

static long long grid_for(long long items, long long per_cta, int n_sm, int per_sm)
{
    long long g = (items + per_cta - 1) / per_cta;
    if (g > (long long)n_sm * per_sm) g = (long long)n_sm * per_sm;
    return g < 1 ? 1 : g;
}

// Tile ranges from the per-tile counts and the scatter of the entries into them.  Returns the
// number of kernels launched.
int launch_bin(const Layout& L, int n_sm, cudaStream_t st)
{
    const long long vt = (long long)L.V * L.T;
    TileRangeOp op{L};
    k_scan<TileRangeOp><<<(unsigned)grid_for(vt, SCAN_TILE, n_sm, 8), SCAN_THREADS, 0, st>>>(
        op, L.scan_lb, L.hdr->ctr + CTR_SCAN_RANGES, L.hdr);
    k_scatter<<<(unsigned)grid_for(L.k_cap, 256, n_sm, 16), 256, 0, st>>>(L);
    return 2;
}

// Per-tile sort (register, shared-memory and long-tile paths).
int launch_tile_sort(const Layout& L, int n_sm, cudaStream_t st)
{
    const long long vt = (long long)L.V * L.T;
    k_tile_sort<<<(unsigned)vt, TS_THREADS, 0, st>>>(L);
    k_tile_sort_large<<<(unsigned)(4 * n_sm), TB_THREADS, 0, st>>>(L);  // four 512-thread CTAs fit an SM
    return 2;
}

}  // namespace cgs
