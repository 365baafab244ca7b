// Stage c of the hot path, after the projection has emitted the (tile, Gaussian) entries and
// the per-tile counts: the depth order inside every tile ("sorted in depth order", Sec. 3.1;
// ties to the lower index).
//
//   tile ranges   single-pass scan of the per-tile counts -> [start, end) of every tile
//   scatter       one thread per entry: a slot in its tile's range (an atomic cursor of one of
//                 the tile's sub-ranges, chosen by the entry's index), key
//                 (FP32 depth bits << 32 | selected index)
//   tile sort     one CTA per tile: up to 128 keys ranked against each other in shared
//                 memory (each key's count of smaller keys is its slot), up to 256 a bitonic
//                 sort held in registers; longer tiles (listed by the range scan) go to a
//                 second kernel, run on a side stream beside the first: up to 512 keys the
//                 register bitonic sort, up to 2048 a stable LSD radix sort in shared memory
//                 over the 8-bit digits of the depth bits that differ within the tile, equal
//                 depths then put in index order; beyond that sorted chunks of 2048 + merge
//                 rounds through global scratch
//
// Within a view, a Gaussian appears at most once per tile, so the 64-bit keys of one tile are
// distinct: the sorted order is exactly (depth, index) whatever order the projection emitted
// the entries in and the scatter placed them.  Every count the sequence needs is read on the
// device; every inter-block wait is bounded and latches ST_SPIN.
#include "common.cuh"
#include "scan.cuh"

namespace cgs {

constexpr int TS_THREADS = 128;
constexpr int RANK_MAX = 2 * TS_THREADS;  // keys per tile sorted by the short-tile kernel

// The start of every (view, tile, sub-range) and the [start, end) of every (view, tile) from the
// per-sub-range counts; tiles longer than RANK_MAX are listed for the long-tile kernel here, so
// that kernel can run beside the short-tile one.  A tile's counts are consecutive items of one
// scanning thread (its SCAN_IPT items start at a multiple of SCAN_IPT, which the sub-range count
// divides), stored in order, so the thread reads back the tile's start at its last sub-range.
struct TileRangeOp {
    Layout L;
    __device__ long long count() const { return ((long long)L.V * L.T) << L.tsub_sh; }
    __device__ uint32_t load(long long i) const { return L.tcnt[i]; }
    __device__ void store(long long i, unsigned long long e, uint32_t x) const
    {
        const long long t = i >> L.tsub_sh;
        const int sub = (int)(i - (t << L.tsub_sh)), last = (1 << L.tsub_sh) - 1;
        L.ssub[i] = (uint32_t)e;
        if (sub == 0) L.ranges[2 * t] = (uint32_t)e;
        if (sub == last) {
            const uint32_t end = (uint32_t)(e + x);
            L.ranges[2 * t + 1] = end;
            if (end - L.ranges[2 * t] > (uint32_t)RANK_MAX) L.big[atomicAdd(&L.hdr->n_big, 1u)] = (uint32_t)t;
        }
    }
    __device__ void finish(unsigned long long total) const { (void)total; }
};
static_assert(SCAN_IPT % TSUB == 0, "a tile's sub-ranges are scanned by one thread");

// One thread per entry: a slot inside its tile's range and the (depth bits, index) key.
__global__ void __launch_bounds__(256) k_scatter(Layout L)
{
    const long long n = entries_kept(L);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const unsigned long long w = L.eraw[k];
        const uint32_t t = (uint32_t)(w >> 32), j = (uint32_t)w;
        const size_t q = ((size_t)t << L.tsub_sh) + (j & ((1u << L.tsub_sh) - 1u));
        const uint32_t slot = L.ssub[q] + atomicAdd(&L.tcur[q], 1u);
        L.ekey[slot] = ((unsigned long long)(uint32_t)L.pkey[j] << 32) | j;
    }
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

constexpr int RANK_ONLY = TS_THREADS;     // up to this many keys by ranking, above by a bitonic sort

// One CTA per (view, tile).  Up to RANK_ONLY keys: every thread ranks one key against all keys
// of the tile in shared memory (n^2 comparisons): first by its 32-bit depth alone (the count of
// strictly smaller depths, four depths per 16-byte load), then, only for a key whose depth
// another key shares (found by counting keys per rank), by index among the equal depths, so
// the rank is the key's slot in (depth, index) order.  Up to RANK_MAX keys: a bitonic sort of
// 256 keys held two per thread (n log^2 n, fewer operations above about 128 keys); longer tiles
// (listed by the range scan) are left to the long-tile kernel, kept apart so the common short
// tiles run at full occupancy.
__global__ void __launch_bounds__(TS_THREADS) k_tile_sort(Layout L)
{
    __shared__ unsigned long long s[RANK_MAX];
    __shared__ __align__(16) uint32_t s_d[RANK_ONLY];  // depth bits
    __shared__ uint32_t s_j[RANK_ONLY], s_c[RANK_ONLY];  // indices; keys per depth rank
    const uint32_t t = blockIdx.x;
    const uint32_t st = L.ranges[2 * (size_t)t], n = L.ranges[2 * (size_t)t + 1] - st;
    if (n == 0 || n > (uint32_t)RANK_MAX) return;  // longer tiles: listed by the range scan
    if (n > (uint32_t)RANK_ONLY) {
        tile_sort_regs<TS_THREADS, 2>(L, s, t, st, n);
        return;
    }
    {
        const uint32_t i = threadIdx.x;
        const uint32_t n4 = (n + 3u) >> 2;
        const unsigned long long key = i < n ? L.ekey[st + i] : ~0ull;
        const uint32_t d = (uint32_t)(key >> 32), j = (uint32_t)key;
        if (i < n) {
            s_d[i] = d;
            s_j[i] = j;
            s_c[i] = 0u;
        } else if (i < 4u * n4) {
            s_d[i] = 0xffffffffu;  // padding: above every depth (positive finite FP32 bits)
        }
        __syncthreads();
        uint32_t r = 0;
        if (i < n) {
            const uint4* d4 = reinterpret_cast<const uint4*>(s_d);
#pragma unroll 4
            for (uint32_t m = 0; m < n4; m++) {
                const uint4 q = d4[m];
                r += (uint32_t)(q.x < d) + (uint32_t)(q.y < d) + (uint32_t)(q.z < d) + (uint32_t)(q.w < d);
            }
            atomicAdd(&s_c[r], 1u);  // keys of equal depth share r
        }
        __syncthreads();
        if (i < n) {
            if (s_c[r] > 1u) {
                // equal depths (rare): ordered by index among themselves
                for (uint32_t m = 0; m < n; m++) r += (uint32_t)(s_d[m] == d && s_j[m] < j);
            }
            L.tval[st + r] = j;
            L.tkey[st + r] = t;
        }
    }
}

// Stable LSD radix sort of n <= RX_CAP keys (FP32 depth bits << 32 | selected index) held in
// shared memory a[] by the CTA (RX_THREADS threads, one digit each in the offset scan); b[] is
// the other buffer.  One pass per 8-bit digit of the depth bits that differ among the keys
// (bits equal in every key cannot change the order): each warp counts the digits of its
// contiguous segment (lanes with the same digit found by __match_any_sync, their leader adds
// the count), the (digit, warp) counts become exclusive offsets in digit-major order, and each
// warp scatters its segment in order, a key's slot being its warp's running offset for the digit
// plus the number of earlier lanes of its group with the same digit.  Equal depths are then put
// in index order (runs of equal depth, rare, sorted by insertion).  Returns the buffer holding
// the sorted keys.
constexpr int RX_THREADS = 256;
constexpr int RX_WARPS = RX_THREADS / 32;
constexpr int RX_CAP = 2048;
constexpr int RX_BITONIC = 512;  // up to this many keys the register bitonic sort is faster (measured)
constexpr size_t RX_SMEM = 2 * RX_CAP * sizeof(unsigned long long) + RX_WARPS * 256 * sizeof(uint32_t);

__device__ unsigned long long* radix_sort_depth(unsigned long long* a, unsigned long long* b, int n,
                                               uint32_t (*hist)[256], uint32_t* s_scan)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    uint32_t orv = 0u, andv = 0xffffffffu;
    for (int i = threadIdx.x; i < n; i += RX_THREADS) {
        const uint32_t d = (uint32_t)(a[i] >> 32);
        orv |= d;
        andv &= d;
    }
    orv = __reduce_or_sync(0xffffffffu, orv);
    andv = __reduce_and_sync(0xffffffffu, andv);
    if (lane == 0) {
        s_scan[warp] = orv;
        s_scan[RX_WARPS + warp] = andv;
    }
    __syncthreads();
    orv = 0u;
    andv = 0xffffffffu;
#pragma unroll
    for (int w = 0; w < RX_WARPS; w++) {
        orv |= s_scan[w];
        andv &= s_scan[RX_WARPS + w];
    }
    const uint32_t vary = orv ^ andv;
    __syncthreads();
    const int seg = (((n + RX_WARPS - 1) / RX_WARPS) + 31) & ~31;
    const int w0 = warp * seg, w1 = min(n, w0 + seg);
    for (int shift = 0; shift < 32; shift += 8) {
        if (((vary >> shift) & 0xffu) == 0u) continue;
        for (int d = lane; d < 256; d += 32) hist[warp][d] = 0u;
        __syncwarp();
        for (int i0 = w0; i0 < w1; i0 += 32) {
            const int i = i0 + lane;
            const bool ok = i < w1;
            const uint32_t d = ok ? ((uint32_t)(a[i] >> 32) >> shift) & 0xffu : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (ok && lane == __ffs(peers) - 1) hist[warp][d] += (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            const int d = threadIdx.x;  // one digit per thread
            uint32_t c[RX_WARPS], sum = 0u;
#pragma unroll
            for (int w = 0; w < RX_WARPS; w++) {
                c[w] = hist[w][d];
                sum += c[w];
            }
            uint32_t tot;
            uint32_t o = block_exclusive_scan<uint32_t>(sum, s_scan, &tot);
#pragma unroll
            for (int w = 0; w < RX_WARPS; w++) {
                hist[w][d] = o;
                o += c[w];
            }
        }
        __syncthreads();
        for (int i0 = w0; i0 < w1; i0 += 32) {
            const int i = i0 + lane;
            const bool ok = i < w1;
            const unsigned long long k = ok ? a[i] : 0ull;
            const uint32_t d = ok ? ((uint32_t)(k >> 32) >> shift) & 0xffu : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0u;
            if (ok && lane == leader) base = hist[warp][d];
            base = __shfl_sync(0xffffffffu, base, leader);
            if (ok) b[base + (uint32_t)__popc(peers & lt)] = k;
            __syncwarp();
            if (ok && lane == leader) hist[warp][d] = base + (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        unsigned long long* tmp = a;
        a = b;
        b = tmp;
    }
    // equal depths in index order (the first key of each run of equal depth sorts the run; the
    // other runs' depths stay where they are while they are sorted)
    bool tie = false;
    for (int i = threadIdx.x; i + 1 < n; i += RX_THREADS) tie |= (a[i] >> 32) == (a[i + 1] >> 32);
    if (__syncthreads_or(tie)) {
        for (int i = threadIdx.x; i < n; i += RX_THREADS) {
            const unsigned long long dv = a[i] >> 32;
            if ((i > 0 && (a[i - 1] >> 32) == dv) || i + 1 >= n || (a[i + 1] >> 32) != dv) continue;
            int e = i + 1;
            while (e < n && (a[e] >> 32) == dv) e++;
            for (int p = i + 1; p < e; p++) {
                const unsigned long long x = a[p];
                int q = p - 1;
                while (q >= i && a[q] > x) {
                    a[q + 1] = a[q];
                    q--;
                }
                a[q + 1] = x;
            }
        }
        __syncthreads();
    }
    return a;
}

// Tiles longer than RANK_MAX: one CTA per listed tile (persistent over the device list).  Up
// to RX_BITONIC keys: the bitonic sort held in registers, two keys per thread; up to RX_CAP: the
// shared-memory radix sort.  Longer: chunks of RX_CAP keys radix-sorted,
// then runs merged pairwise through global scratch (the entry buffer, free after the scatter);
// with distinct keys, an element's output position is its rank in its own run plus the number
// of smaller keys in the other run.
__global__ void __launch_bounds__(RX_THREADS) k_tile_sort_large(Layout L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* sa = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* sb = sa + RX_CAP;
    uint32_t(*hist)[256] = reinterpret_cast<uint32_t(*)[256]>(sb + RX_CAP);
    __shared__ uint32_t s_scan[33];
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
        if (n <= (uint32_t)RX_BITONIC) {
            tile_sort_regs<RX_THREADS, RX_BITONIC / RX_THREADS>(L, sa, t, st, n);
            __syncthreads();
            continue;
        }
        if (n <= (uint32_t)RX_CAP) {
            for (uint32_t i = threadIdx.x; i < n; i += RX_THREADS) sa[i] = L.ekey[st + i];
            __syncthreads();
            const unsigned long long* r = radix_sort_depth(sa, sb, (int)n, hist, s_scan);
            for (uint32_t i = threadIdx.x; i < n; i += RX_THREADS) {
                L.tval[st + i] = (uint32_t)r[i];
                L.tkey[st + i] = t;
            }
            __syncthreads();
            continue;
        }
        unsigned long long* a = L.ekey + st;
        unsigned long long* b = L.eraw + st;
        for (uint32_t c0 = 0; c0 < n; c0 += RX_CAP) {
            const int m = (int)min((uint32_t)RX_CAP, n - c0);
            for (int i = threadIdx.x; i < m; i += RX_THREADS) sa[i] = a[c0 + i];
            __syncthreads();
            const unsigned long long* r = radix_sort_depth(sa, sb, m, hist, s_scan);
            for (int i = threadIdx.x; i < m; i += RX_THREADS) a[c0 + i] = r[i];
            __syncthreads();
        }
        for (uint32_t width = RX_CAP; width < n; width <<= 1) {
            for (uint32_t i = threadIdx.x; i < n; i += RX_THREADS) {
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
        for (uint32_t i = threadIdx.x; i < n; i += RX_THREADS) {
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
    k_scan<TileRangeOp><<<(unsigned)grid_for(vt << L.tsub_sh, SCAN_TILE, n_sm, 8), SCAN_THREADS, 0, st>>>(
        op, L.scan_lb, L.hdr->ctr + CTR_SCAN_RANGES, L.hdr);
    k_scatter<<<(unsigned)grid_for(L.k_cap, 256, n_sm, 16), 256, 0, st>>>(L);
    return 2;
}

// A second stream and two events, per host thread and device, on which the long-tile sort runs
// beside the short-tile sort (fork after the scatter, join before the compositing).  Created on
// first use outside a stream capture; until then the two kernels run one after the other.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    bool ok = false, tried = false;
};

static SideStream* side_stream(cudaStream_t st)
{
    constexpr int MAX_DEV = 64;
    static thread_local SideStream side[MAX_DEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return nullptr;
    SideStream& x = side[dev];
    if (!x.tried) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
        x.tried = true;
        // relaxed for this thread while creating, so a capture running on another thread's
        // stream is not disturbed
        cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
        cudaThreadExchangeStreamCaptureMode(&mode);
        x.ok = cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) == cudaSuccess;
        cudaThreadExchangeStreamCaptureMode(&mode);
    }
    return x.ok ? &x : nullptr;
}

// Per-tile sort (register, shared-memory and long-tile paths).  Returns the number of kernels
// launched, or -1 if the fork or join of the side stream failed.
int launch_tile_sort(const Layout& L, int n_sm, cudaStream_t st)
{
    const long long vt = (long long)L.V * L.T;
    static bool smem_set[64] = {};  // the long-tile kernel's dynamic shared memory, set once per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !smem_set[dev]) {
        cudaFuncSetAttribute(k_tile_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RX_SMEM);
        smem_set[dev] = true;
    }
    SideStream* sd = side_stream(st);
    if (sd && cudaEventRecord(sd->fork, st) == cudaSuccess && cudaStreamWaitEvent(sd->s, sd->fork, 0) == cudaSuccess) {
        k_tile_sort_large<<<(unsigned)(5 * n_sm), RX_THREADS, RX_SMEM, sd->s>>>(L);  // five 40-KB CTAs fit an SM
        k_tile_sort<<<(unsigned)vt, TS_THREADS, 0, st>>>(L);
        if (cudaEventRecord(sd->join, sd->s) != cudaSuccess || cudaStreamWaitEvent(st, sd->join, 0) != cudaSuccess)
            return -1;
        return 2;
    }
    k_tile_sort<<<(unsigned)vt, TS_THREADS, 0, st>>>(L);
    k_tile_sort_large<<<(unsigned)(5 * n_sm), RX_THREADS, RX_SMEM, st>>>(L);
    return 2;
}

}  // namespace cgs
