// Stage c of the hot path: compaction of the visible Gaussians, a stable LSD radix sort by
// (view, depth), duplication into (view * tiles + tile, Gaussian) entries in that depth
// order, a stable radix sort by tile, and the per-tile ranges.  The tile sort is stable, so
// entries of one tile stay in (depth, index) order: the list each tile composites is
// "sorted in depth order" (Sec. 3.1) with ties to the lower index.
//
// All device-count dependent kernels are persistent grids that read the count on the
// device, so the whole sequence runs without a host round trip.  Passes over keys are
// single-pass (decoupled look-back) kernels; every wait on another block is bounded and
// latches ST_SPIN instead of hanging.
#include "common.cuh"

namespace cgs {

constexpr uint32_t LB_AGG = 1u << 30, LB_INC = 2u << 30, LB_FLAGS = 3u << 30;

template <typename K>
struct SortTraits;
template <>
struct SortTraits<uint32_t> { static constexpr int IPT = 12; };
template <>
struct SortTraits<unsigned long long> { static constexpr int IPT = 8; };

long long sort_tile_items(int key_bytes) { return 256LL * (key_bytes == 4 ? 12 : 8); }

// Digit histograms of every pass in one read of the keys; also clears the look-back
// words the first pass will use.
template <typename K>
__global__ void __launch_bounds__(256) k_sort_hist(const K* __restrict__ keys, const uint32_t* n_ptr, long long n_cap,
                                                   uint32_t* hist, int passes, uint32_t* lb0)
{
    __shared__ uint32_t sh[MAX_DEPTH_PASSES * 256];
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    long long n = *n_ptr;
    if (n > n_cap) n = n_cap;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += warps * 32) {
        const long long i = base + lane;
        const bool valid = i < n;
        const K k = valid ? keys[i] : K(0);
        for (int p = 0; p < passes; p++) {
            const uint32_t d = valid ? (uint32_t)(k >> (8 * p)) & 255u : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&sh[p * 256 + d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
    const long long tile = 256LL * SortTraits<K>::IPT;
    const long long words = ((n + tile - 1) / tile) * 256;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (long long)gridDim.x * blockDim.x)
        lb0[i] = 0;
}

// One stable counting pass on the 8-bit digit at `shift`.
template <typename K>
__global__ void __launch_bounds__(256) k_onesweep(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* kout,
                                                  uint32_t* vout, const uint32_t* n_ptr, long long n_cap,
                                                  const uint32_t* hist, uint32_t* lb, uint32_t* lb_next,
                                                  uint32_t* tile_ctr, Header* hdr, int shift)
{
    constexpr int IPT = SortTraits<K>::IPT;
    constexpr int TILE = 256 * IPT;
    constexpr int NW = 8;
    __shared__ uint32_t s_glob[256];
    __shared__ uint32_t s_whist[NW][256];
    __shared__ uint32_t s_texcl[256];
    __shared__ uint32_t s_pos[256];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_tile;
    __shared__ K s_k[TILE];
    __shared__ uint32_t s_v[TILE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long n = *n_ptr;
    if (n > n_cap) n = n_cap;
    const long long n_tiles = (n + TILE - 1) / TILE;
    {
        uint32_t tot;
        s_glob[tid] = block_exclusive_scan<uint32_t>(hist[tid], s_scan, &tot);
    }
    while (true) {
        if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
        for (int i = tid; i < NW * 256; i += 256) (&s_whist[0][0])[i] = 0;
        __syncthreads();
        const long long t = s_tile;
        if (t >= n_tiles) break;
        if (lb_next) lb_next[t * 256 + tid] = 0;
        const long long base = t * TILE;
        K k[IPT];
        uint32_t val[IPT], d[IPT], rk[IPT];
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            const long long pos = base + (long long)warp * 32 * IPT + j * 32 + lane;
            const bool valid = pos < n;
            k[j] = valid ? kin[pos] : K(0);
            val[j] = valid ? vin[pos] : 0u;
            d[j] = valid ? ((uint32_t)(k[j] >> shift) & 255u) : 256u;
        }
        // stable rank inside the warp's contiguous sub-range: items are ordered (j, lane)
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            const uint32_t peers = __match_any_sync(0xffffffffu, d[j]);
            const uint32_t below = __popc(peers & lanemask_lt());
            const uint32_t before = d[j] < 256u ? s_whist[warp][d[j]] : 0u;
            rk[j] = before + below;
            __syncwarp();
            if (d[j] < 256u && below == 0) s_whist[warp][d[j]] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const uint32_t c = s_whist[w][tid];
            s_whist[w][tid] = cnt;
            cnt += c;
        }
        uint32_t* my = lb + t * 256 + tid;
        st_volatile(my, (t == 0 ? LB_INC : LB_AGG) | cnt);
        uint32_t tot;
        const uint32_t tex = block_exclusive_scan<uint32_t>(cnt, s_scan, &tot);
        s_texcl[tid] = tex;
        uint32_t excl = 0;
        if (t > 0) {
            long long p = t - 1;
            while (true) {
                uint32_t w;
                int spins = 0;
                while (true) {
                    w = ld_volatile(lb + p * 256 + tid);
                    if (w & LB_FLAGS) break;
                    if (++spins > SPIN_LIMIT) {
                        latch(hdr, ST_SPIN);
                        atomicAdd(&hdr->spin_giveups, 1u);
                        w = LB_INC;
                        break;
                    }
                    __nanosleep(64);
                }
                excl += w & ~LB_FLAGS;
                if ((w & LB_FLAGS) == LB_INC || p == 0) break;
                --p;
            }
            st_volatile(my, LB_INC | (excl + cnt));
        }
        s_pos[tid] = s_glob[tid] + excl - tex;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < IPT; j++) {
            if (d[j] < 256u) {
                const uint32_t lp = s_texcl[d[j]] + s_whist[warp][d[j]] + rk[j];
                s_k[lp] = k[j];
                s_v[lp] = val[j];
            }
        }
        __syncthreads();
        const int tile_n = (int)((n - base) < TILE ? (n - base) : TILE);
        for (int i = tid; i < tile_n; i += 256) {
            const K key = s_k[i];
            const uint32_t o = s_pos[(uint32_t)(key >> shift) & 255u] + (uint32_t)i;
            kout[o] = key;
            vout[o] = s_v[i];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// single-pass exclusive scan with a per-item action (decoupled look-back, u64 totals)
// ---------------------------------------------------------------------------------------
constexpr unsigned long long SF_AGG = 1ull << 62, SF_INC = 2ull << 62, SF_FLAGS = 3ull << 62;

template <class Op>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(Op op, unsigned long long* lb, uint32_t* tile_ctr, Header* hdr)
{
    __shared__ unsigned long long s_buf[33];
    __shared__ unsigned long long s_prefix;
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x;
    const long long n = op.count();
    const long long n_tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    while (true) {
        if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
        __syncthreads();
        const long long t = s_tile;
        if (t >= n_tiles) break;
        const long long base = t * SCAN_TILE + (long long)tid * SCAN_IPT;
        uint32_t x[SCAN_IPT];
        unsigned long long sum = 0;
#pragma unroll
        for (int j = 0; j < SCAN_IPT; j++) {
            x[j] = (base + j < n) ? op.load(base + j) : 0u;
            sum += x[j];
        }
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_scan<unsigned long long>(sum, s_buf, &tot);
        if (tid < 32) {
            // warp-parallel look-back: lane l inspects tile p - l; the window slides back by 32
            // until a tile with an inclusive prefix is found
            const int lane = tid;
            if (lane == 0) st_volatile64(&lb[t], (t == 0 ? SF_INC : SF_AGG) | tot);
            unsigned long long excl = 0;
            long long p = t - 1;
            while (p >= 0) {
                const long long q = p - lane;
                unsigned long long w = SF_INC;  // before tile 0: an inclusive zero
                if (q >= 0) {
                    int spins = 0;
                    while (true) {
                        w = ld_volatile64(&lb[q]);
                        if (w & SF_FLAGS) break;
                        if (++spins > SPIN_LIMIT) {
                            latch(hdr, ST_SPIN);
                            atomicAdd(&hdr->spin_giveups, 1u);
                            w = SF_INC;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                const uint32_t inc = __ballot_sync(0xffffffffu, (w & SF_FLAGS) == SF_INC);
                const int stop = inc ? __ffs(inc) - 1 : 31;
                unsigned long long val = lane <= stop ? (w & ~SF_FLAGS) : 0ull;
#pragma unroll
                for (int o = 16; o; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                excl += val;
                if (inc) break;
                p -= 32;
            }
            if (lane == 0) {
                if (t > 0) st_volatile64(&lb[t], SF_INC | (excl + tot));
                s_prefix = excl;
                if (t == n_tiles - 1) op.finish(excl + tot);
            }
        }
        __syncthreads();
        unsigned long long run = s_prefix + ex;
#pragma unroll
        for (int j = 0; j < SCAN_IPT; j++) {
            if (base + j < n) op.store(base + j, run, x[j]);
            run += x[j];
        }
        __syncthreads();
    }
}

// Keeps the selected Gaussians with tiles_touched > 0, in selected-index order.
struct CompactOp {
    Layout L;
    __device__ long long count() const { return L.hdr->n_sel; }
    __device__ uint32_t load(long long j) const { return L.tt[j] > 0 ? 1u : 0u; }
    __device__ void store(long long j, unsigned long long e, uint32_t x) const
    {
        if (x) {
            L.dkey[0][e] = L.pkey[j];
            L.dval[0][e] = (uint32_t)j;
        }
    }
    __device__ void finish(unsigned long long total) const { L.hdr->n_vis = (uint32_t)total; }
};

// Exclusive offsets of the tile entries of the (view, depth)-sorted visible Gaussians.
struct OffsetOp {
    Layout L;
    const uint32_t* dval;
    __device__ long long count() const { return L.hdr->n_vis; }
    __device__ uint32_t load(long long r) const { return L.tt[dval[r]]; }
    __device__ void store(long long r, unsigned long long e, uint32_t x) const
    {
        (void)x;
        L.offs[r] = (uint32_t)(e < 0xffffffffull ? e : 0xffffffffull);
    }
    __device__ void finish(unsigned long long total) const
    {
        L.hdr->k_total = total;
        const unsigned long long cap = (unsigned long long)L.k_cap;
        L.hdr->k_used = (uint32_t)(total < cap ? total : cap);
        if (total > cap) latch(L.hdr, ST_CAPACITY);
    }
};

// Duplication, one thread per output entry k: the owning Gaussian is the last r with
// offs[r] <= k (binary search), the tile is the (k - offs[r])-th of its rect in row-major
// order.  Entries come out in (view, depth, index) order, tiles row-major inside a rect.
__global__ void __launch_bounds__(256) k_emit(Layout L, const unsigned long long* __restrict__ dkey,
                                              const uint32_t* __restrict__ dval)
{
    const long long n = L.hdr->k_used;
    const uint32_t nv = L.hdr->n_vis;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nv;  // offs[lo] <= k < offs[hi] (offs[nv] taken as +inf)
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if ((long long)L.offs[mid] <= k) lo = mid; else hi = mid;
        }
        const uint32_t j = dval[lo];
        const uint32_t view = (uint32_t)(dkey[lo] >> 32);
        const uint2 rc = L.rect[j];
        const uint32_t tx0 = rc.x & 0xffffu, ty0 = rc.x >> 16, w = (rc.y & 0xffffu) - tx0;
        const uint32_t local = (uint32_t)(k - (long long)L.offs[lo]);
        const uint32_t ty = ty0 + local / w, tx = tx0 + local % w;
        L.tkey[0][k] = view * (uint32_t)L.T + ty * (uint32_t)L.tiles_x + tx;
        L.tval[0][k] = j;
    }
}

// [start, end) of every (view, tile) key in the sorted entries; ranges were cleared.
__global__ void k_ranges(const uint32_t* __restrict__ keys, const Header* hdr, uint32_t* ranges)
{
    const long long n = hdr->k_used;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const uint32_t k = keys[r];
        if (r == 0 || keys[r - 1] != k) ranges[2 * (size_t)k] = (uint32_t)r;
        if (r == n - 1 || keys[r + 1] != k) ranges[2 * (size_t)k + 1] = (uint32_t)(r + 1);
    }
}

template <typename K>
static void radix_sort(K* const keys[2], uint32_t* const vals[2], const uint32_t* n_ptr, long long n_cap, uint32_t* hist,
                       int passes, uint32_t* const lb[2], uint32_t* ctr, Header* hdr, int n_sm, cudaStream_t st)
{
    const long long tile = 256LL * SortTraits<K>::IPT;
    const long long tiles = (n_cap + tile - 1) / tile;
    long long hg = (n_cap + 255) / 256;
    if (hg > (long long)n_sm * 4) hg = (long long)n_sm * 4;
    if (hg < 1) hg = 1;
    k_sort_hist<K><<<(unsigned)hg, 256, 0, st>>>(keys[0], n_ptr, n_cap, hist, passes, lb[0]);
    long long grid = tiles < (long long)n_sm * 4 ? tiles : (long long)n_sm * 4;
    if (grid < 1) grid = 1;
    for (int p = 0; p < passes; p++) {
        const int a = p & 1;
        k_onesweep<K><<<(unsigned)grid, 256, 0, st>>>(keys[a], vals[a], keys[a ^ 1], vals[a ^ 1], n_ptr, n_cap,
                                                      hist + 256 * p, lb[a], p + 1 < passes ? lb[a ^ 1] : nullptr,
                                                      ctr + p, hdr, 8 * p);
    }
}

static long long grid_for(long long items, long long per_cta, int n_sm, int per_sm)
{
    long long g = (items + per_cta - 1) / per_cta;
    if (g > (long long)n_sm * per_sm) g = (long long)n_sm * per_sm;
    return g < 1 ? 1 : g;
}

// Visible compaction in selected-index order.  Returns the number of kernels launched.
int launch_compact(const Layout& L, int n_sm, cudaStream_t st)
{
    CompactOp cop{L};
    k_scan<CompactOp><<<(unsigned)grid_for(L.n_cap, SCAN_TILE, n_sm, 8), SCAN_THREADS, 0, st>>>(
        cop, L.scan_lb, L.hdr->ctr + CTR_SCAN_COMPACT, L.hdr);
    return 1;
}

// Stable (view, depth) radix sort of the compacted visible Gaussians.
int launch_depth_sort(const Layout& L, int n_sm, cudaStream_t st)
{
    radix_sort<unsigned long long>(L.dkey, L.dval, &L.hdr->n_vis, L.n_cap, L.hist_depth, L.depth_passes, L.lb,
                                   L.hdr->ctr + CTR_DEPTH_PASS0, L.hdr, n_sm, st);
    return 1 + L.depth_passes;
}

// Offsets of every visible Gaussian's entries, then duplication into tile entries.
int launch_emit_stage(const Layout& L, int n_sm, cudaStream_t st)
{
    const long long scan_tiles = (L.n_cap + SCAN_TILE - 1) / SCAN_TILE;
    OffsetOp oop{L, L.dval[L.depth_sorted]};
    k_scan<OffsetOp><<<(unsigned)grid_for(L.n_cap, SCAN_TILE, n_sm, 8), SCAN_THREADS, 0, st>>>(
        oop, L.scan_lb + scan_tiles, L.hdr->ctr + CTR_SCAN_EMIT, L.hdr);
    k_emit<<<(unsigned)grid_for(L.k_cap, 256, n_sm, 16), 256, 0, st>>>(L, L.dkey[L.depth_sorted],
                                                                       L.dval[L.depth_sorted]);
    return 2;
}

// Stable sort by tile (keeps the depth order inside each tile) and the per-tile ranges.
int launch_tile_stage(const Layout& L, int n_sm, cudaStream_t st)
{
    radix_sort<uint32_t>(L.tkey, L.tval, &L.hdr->k_used, L.k_cap, L.hist_tile, L.tile_passes, L.lb,
                         L.hdr->ctr + CTR_TILE_PASS0, L.hdr, n_sm, st);
    k_ranges<<<(unsigned)grid_for(L.k_cap, 256, n_sm, 8), 256, 0, st>>>(L.tkey[L.tile_sorted], L.hdr, L.ranges);
    return 2 + L.tile_passes;
}

}  // namespace cgs
