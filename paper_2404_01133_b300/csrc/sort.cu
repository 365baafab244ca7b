// Stage c of the hot path, after the projection has emitted the (tile, Gaussian) entries and
// the per-tile counts: the depth order inside every tile ("sorted in depth order", Sec. 3.1;
// ties to the lower index).
//
//   tile ranges   single-pass scan of the per-tile counts -> [start, end) of every tile
//   scatter       one thread per entry: a slot in its tile's range (atomic cursor), key
//                 (FP32 depth bits << 32 | selected index)
//   tile sort     one CTA per tile: up to 256 keys ranked against each other in shared
//                 memory (each key's count of smaller keys is its slot); longer tiles go to a
//                 second kernel: up to 2048 keys a bitonic sort held in registers (shuffles
//                 within warps, shared memory only for the strides that cross warps), up to
//                 4096 a bitonic sort in shared memory, beyond that sorted chunks + merge
//                 rounds through global scratch
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

constexpr int TS_THREADS = 128;
constexpr int TS_CAP = 2048;  // keys per tile sorted in registers by the long-tile kernel
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

// Ascending bitonic sort of np = THREADS * E keys held by the CTA in registers: warp w
// holds keys [32 E w, 32 E (w + 1)), lane l's x[e] being key 32 E w + 32 e + l.  Exchanges
// between lanes of a warp are shuffles, between a lane's own registers are moves; only the
// strides that cross warps go through shared memory (a store, one synchronised pass per
// stride, a load), so a sort of 2048 keys takes 6 shared-memory passes instead of 66.
template <int THREADS, int E>
__device__ __forceinline__ void cta_bitonic(unsigned long long (&x)[E], unsigned long long* s)
{
    constexpr int NP = THREADS * E, WS = 32 * E;
    const int lane = threadIdx.x & 31;
    const int base = (threadIdx.x >> 5) * WS;
#pragma unroll
    for (int size = 2; size <= NP; size <<= 1) {
        int stride = size >> 1;
        if (stride >= WS) {
#pragma unroll
            for (int e = 0; e < E; e++) s[base + 32 * e + lane] = x[e];
            __syncthreads();
            for (; stride >= WS; stride >>= 1) {
                for (int i = threadIdx.x; i < NP / 2; i += THREADS) {
                    const int lo = 2 * i - (i & (stride - 1));
                    const int hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const unsigned long long a = s[lo], b = s[hi];
                    if ((a > b) == up) { s[lo] = b; s[hi] = a; }
                }
                __syncthreads();
            }
#pragma unroll
            for (int e = 0; e < E; e++) x[e] = s[base + 32 * e + lane];
            __syncthreads();
        }
#pragma unroll
        for (int d = WS / 2; d > 0; d >>= 1) {
            if (d > stride) continue;
#pragma unroll
            for (int e = 0; e < E; e++) {
                const bool up = ((base + 32 * e + lane) & size) == 0;
                if (d >= 32) {
                    const int pe = e ^ (d >> 5);
                    if (pe > e) {
                        const unsigned long long a = x[e], b = x[pe];
                        const bool sw = (a > b) == up;
                        x[e] = sw ? b : a;
                        x[pe] = sw ? a : b;
                    }
                } else {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x[e], d);
                    const unsigned long long mn = x[e] < y ? x[e] : y, mx = x[e] < y ? y : x[e];
                    x[e] = (((lane & d) == 0) == up) ? mn : mx;
                }
            }
        }
    }
}

template <int THREADS, int E>
__device__ __forceinline__ void tile_sort_regs(const Layout& L, unsigned long long* s, uint32_t t, uint32_t st,
                                               uint32_t n)
{
    constexpr int WS = 32 * E;
    const int lane = threadIdx.x & 31;
    const int base = (threadIdx.x >> 5) * WS;
    unsigned long long x[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t i = (uint32_t)(base + 32 * e + lane);
        x[e] = i < n ? L.ekey[st + i] : ~0ull;
    }
    cta_bitonic<THREADS, E>(x, s);
#pragma unroll
    for (int e = 0; e < E; e++) {
        const uint32_t i = (uint32_t)(base + 32 * e + lane);
        if (i < n) {
            L.tval[st + i] = (uint32_t)x[e];
            L.tkey[st + i] = t;
        }
    }
}

constexpr int RANK_MAX = 2 * TS_THREADS;  // keys per tile sorted by this kernel
constexpr int RANK_ONLY = TS_THREADS;     // up to this many keys by ranking, above by a bitonic sort

// One CTA per (view, tile).  Up to RANK_ONLY keys: every thread ranks one key against all keys
// of the tile in shared memory (keys are distinct, so the rank is the output slot; n^2
// comparisons); up to RANK_MAX keys: a bitonic sort of 256 keys held two per thread (n log^2 n,
// fewer operations above about 128 keys); longer tiles are listed for the long-tile kernel,
// kept apart so the common short tiles run at full occupancy.
__global__ void __launch_bounds__(TS_THREADS) k_tile_sort(Layout L)
{
    __shared__ unsigned long long s[RANK_MAX];
    const uint32_t t = blockIdx.x;
    const uint32_t st = L.ranges[2 * (size_t)t], n = L.ranges[2 * (size_t)t + 1] - st;
    if (n == 0) return;
    if (n > (uint32_t)RANK_MAX) {
        if (threadIdx.x == 0) L.big[atomicAdd(&L.hdr->n_big, 1u)] = t;
        return;
    }
    if (n > (uint32_t)RANK_ONLY) {
        tile_sort_regs<TS_THREADS, 2>(L, s, t, st, n);
        return;
    }
    {
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
    }
}

// Tiles longer than RANK_MAX: one CTA per listed tile (persistent over the device list).  Up
// to TS_CAP keys: bitonic sort held in registers (cta_bitonic).  Longer: chunks of LT_CAP keys
// sorted in shared memory (the whole tile when it fits), then runs merged pairwise through
// global scratch (the entry buffer, free after the scatter); with distinct keys, an element's
// output position is its rank in its own run plus the number of smaller keys in the other
// run.
constexpr int TB_THREADS = 256;
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
        if (n <= (uint32_t)TS_CAP) {
            // listed tiles hold more than 256 keys: two, four or eight keys per thread
            if (n <= 2u * TB_THREADS) tile_sort_regs<TB_THREADS, 2>(L, s, t, st, n);
            else if (n <= 4u * TB_THREADS) tile_sort_regs<TB_THREADS, 4>(L, s, t, st, n);
            else tile_sort_regs<TB_THREADS, 8>(L, s, t, st, n);
            __syncthreads();
            continue;
        }
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
    k_tile_sort_large<<<(unsigned)(6 * n_sm), TB_THREADS, 0, st>>>(L);  // six 256-thread CTAs fit an SM
    return 2;
}

}  // namespace cgs
