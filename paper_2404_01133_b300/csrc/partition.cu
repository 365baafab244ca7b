// Block partition of a Gaussian scene (Sec. 3.2.2) and the block of a camera pose (Eq. 4).
//
//   normalisation   h = 2 (p - p_min) / (p_max - p_min) - 1 per axis: the foreground box
//                   maps to [-1, 1]^3
//   contraction     Eq. 2: h when ||h||_inf <= 1, else (2 - 1/||h||_inf) h / ||h||_inf
//   grid            the contracted cube (-2, 2)^3 split evenly: along an axis of g cells the
//                   inner bounds are b_i = 4 i / g - 2 and a coordinate c lies in cell i when
//                   b_i <= c < b_{i+1}; the outer cells are open to -inf / +inf
//   block           ix + g_x (iy + g_y iz); -1 when the contracted point is not finite
//   grouping        a stable counting sort by block: perm lists block 0's Gaussians in scene
//                   order, then block 1's, ...
//
// Every value that decides a block is FP32 with one rounding per operation in the order
// above (this file is compiled without FMA contraction).
//
// Grouping is two passes over warp-owned chunks of CH consecutive Gaussians:
//   k_part_assign   block of every Gaussian and, per chunk, a block histogram (warp-private
//                   shared-memory counters) written to cnt[block][chunk]
//   k_scan          exclusive scan of cnt in (block, chunk) order: the first grouped position
//                   of every (block, chunk); block offsets fall out at chunk 0
//   k_part_scatter  every warp walks its chunk again in scene order; a Gaussian's position is
//                   its chunk's running counter for its block plus its rank among the earlier
//                   lanes of the warp with the same block -- so the order is stable
// and a gather (k_gather_rows) moves attribute rows into the grouped order.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "scan.cuh"

namespace cgs {

constexpr int PART_WARPS = 8;
constexpr int PART_THREADS = 32 * PART_WARPS;
constexpr int PART_MIN_CHUNK = 1024;
constexpr int PART_ILP = 8;  // groups of 32 loaded before any is used
constexpr long long PART_MAX_COUNTS = 1ll << 23;  // bound on blocks x chunks

struct PartParams {
    float pmin[3], pmax[3];
    int g[3];
    int nb;
    float bnd[3][CGS_PARTITION_MAX_CELLS + 1];  // bnd[a][i] = b_i, i = 1 .. g-1
};

__device__ __forceinline__ void contract_point(const PartParams& P, float x, float y, float z, float c[3])
{
    const float p[3] = {x, y, z};
    float h[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float d = __fsub_rn(p[a], P.pmin[a]);
        const float e = __fsub_rn(P.pmax[a], P.pmin[a]);
        const float q = __fdiv_rn(__fmul_rn(2.0f, d), e);
        h[a] = __fsub_rn(q, 1.0f);
    }
    float m = fabsf(h[0]);
    if (fabsf(h[1]) > m) m = fabsf(h[1]);
    if (fabsf(h[2]) > m) m = fabsf(h[2]);
    if (m <= 1.0f) {
        c[0] = h[0]; c[1] = h[1]; c[2] = h[2];
        return;
    }
    const float s = __fsub_rn(2.0f, __fdiv_rn(1.0f, m));
#pragma unroll
    for (int a = 0; a < 3; a++) c[a] = __fmul_rn(s, __fdiv_rn(h[a], m));
}

// Cell of c along axis a: an estimate from the cell width, then moved until
// bnd[k] <= c < bnd[k+1] holds exactly against the stored bounds.
__device__ __forceinline__ int axis_cell(const float* bnd, int g, float c)
{
    int k = (int)floorf((c + 2.0f) * (0.25f * (float)g));
    k = k < 0 ? 0 : (k > g - 1 ? g - 1 : k);
    while (k < g - 1 && bnd[k + 1] <= c) k++;
    while (k > 0 && bnd[k] > c) k--;
    return k;
}

__device__ __forceinline__ int point_block(const PartParams& P, const float* sb, float x, float y, float z)
{
    float c[3];
    contract_point(P, x, y, z, c);
    if (!(isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2]))) return -1;
    const int ix = axis_cell(sb, P.g[0], c[0]);
    const int iy = axis_cell(sb + (CGS_PARTITION_MAX_CELLS + 1), P.g[1], c[1]);
    const int iz = axis_cell(sb + 2 * (CGS_PARTITION_MAX_CELLS + 1), P.g[2], c[2]);
    return ix + P.g[0] * (iy + P.g[1] * iz);
}

__device__ __forceinline__ void load_bounds(const PartParams& P, float* sb)
{
    for (int i = threadIdx.x; i < 3 * (CGS_PARTITION_MAX_CELLS + 1); i += blockDim.x)
        sb[i] = (&P.bnd[0][0])[i];
    __syncthreads();
}

// Contracted positions (and nothing else), one thread per point.
__global__ void __launch_bounds__(256) k_contract(PartParams P, const float* __restrict__ pos, long long stride,
                                                  long long n, float* __restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float* r = pos + i * stride;
        float c[3];
        contract_point(P, __ldg(r), __ldg(r + 1), __ldg(r + 2), c);
        out[3 * i] = c[0];
        out[3 * i + 1] = c[1];
        out[3 * i + 2] = c[2];
    }
}

// Block of every point, one thread per point (camera poses, Eq. 4).
__global__ void __launch_bounds__(256) k_point_blocks(PartParams P, const float* __restrict__ pos, long long stride,
                                                      long long n, int32_t* __restrict__ block)
{
    __shared__ float sb[3 * (CGS_PARTITION_MAX_CELLS + 1)];
    load_bounds(P, sb);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float* r = pos + i * stride;
        block[i] = point_block(P, sb, __ldg(r), __ldg(r + 1), __ldg(r + 2));
    }
}

// Pass 1: blocks and per-chunk histograms.  Warp w of the grid owns chunks w, w + W, ...; it
// loads PART_ILP groups of 32 positions before computing any block (memory parallelism) and
// counts blocks in warp-private shared-memory counters.
__global__ void __launch_bounds__(PART_THREADS) k_part_assign(PartParams P, const float* __restrict__ pos,
                                                             long long stride, long long n, long long ch,
                                                             long long n_chunks, int32_t* __restrict__ block,
                                                             uint32_t* __restrict__ cnt)
{
    extern __shared__ uint32_t s_hist[];  // [PART_WARPS][nb]
    __shared__ float sb[3 * (CGS_PARTITION_MAX_CELLS + 1)];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* hist = s_hist + warp * P.nb;
    for (int b = lane; b < P.nb; b += 32) hist[b] = 0;
    load_bounds(P, sb);
    const long long gw = (long long)blockIdx.x * PART_WARPS + warp, nw = (long long)gridDim.x * PART_WARPS;
    for (long long chunk = gw; chunk < n_chunks; chunk += nw) {
        const long long c0 = chunk * ch, c1 = min(n, c0 + ch);
        for (long long base = c0; base < c1; base += 32 * PART_ILP) {
            float x[PART_ILP], y[PART_ILP], z[PART_ILP];
#pragma unroll
            for (int u = 0; u < PART_ILP; u++) {
                const long long i = base + u * 32 + lane;
                x[u] = y[u] = z[u] = 0.0f;
                if (i < c1) {
                    const float* r = pos + i * stride;
                    x[u] = __ldg(r);
                    y[u] = __ldg(r + 1);
                    z[u] = __ldg(r + 2);
                }
            }
#pragma unroll
            for (int u = 0; u < PART_ILP; u++) {
                const long long i = base + u * 32 + lane;
                if (i < c1) {
                    const int b = point_block(P, sb, x[u], y[u], z[u]);
                    block[i] = b;
                    if (b >= 0) atomicAdd(&hist[b], 1u);
                }
            }
        }
        __syncwarp();
        for (int b = lane; b < P.nb; b += 32) {
            cnt[(long long)b * n_chunks + chunk] = hist[b];
            hist[b] = 0;
        }
        __syncwarp();
    }
}

// Scan of cnt in (block, chunk) order, in place; offsets of the blocks.
struct PartScanOp {
    uint32_t* cnt;
    long long n_chunks;
    long long total;
    int64_t* offset;
    __device__ long long count() const { return total; }
    __device__ uint32_t load(long long t) const { return cnt[t]; }
    __device__ void store(long long t, unsigned long long e, uint32_t x) const
    {
        (void)x;
        cnt[t] = (uint32_t)e;
        if (t % n_chunks == 0) offset[t / n_chunks] = (int64_t)e;
    }
    __device__ void finish(unsigned long long tot) const { offset[total / n_chunks] = (int64_t)tot; }
};

// Pass 2: stable scatter of scene indices into their grouped positions.  The block ids of
// PART_ILP groups are loaded first, then ranked group by group in chunk order.
__global__ void __launch_bounds__(PART_THREADS) k_part_scatter(int nb, long long n, long long ch, long long n_chunks,
                                                              const int32_t* __restrict__ block,
                                                              const uint32_t* __restrict__ base,
                                                              int32_t* __restrict__ perm, int32_t* __restrict__ rank)
{
    extern __shared__ uint32_t s_run[];  // [PART_WARPS][nb]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* run = s_run + warp * nb;
    const uint32_t lt = (1u << lane) - 1u;
    const long long gw = (long long)blockIdx.x * PART_WARPS + warp, nw = (long long)gridDim.x * PART_WARPS;
    for (long long chunk = gw; chunk < n_chunks; chunk += nw) {
        for (int b = lane; b < nb; b += 32) run[b] = __ldg(base + (long long)b * n_chunks + chunk);
        __syncwarp();
        const long long c0 = chunk * ch, c1 = min(n, c0 + ch);
        for (long long b0 = c0; b0 < c1; b0 += 32 * PART_ILP) {
            int bl[PART_ILP];
#pragma unroll
            for (int u = 0; u < PART_ILP; u++) {
                const long long i = b0 + u * 32 + lane;
                bl[u] = i < c1 ? __ldg(block + i) : -1;
            }
#pragma unroll
            for (int u = 0; u < PART_ILP; u++) {
                const long long i = b0 + u * 32 + lane;
                const int b = bl[u];
                const uint32_t peers = __match_any_sync(0xffffffffu, b);
                uint32_t slot = 0;
                if (b >= 0) slot = run[b] + __popc(peers & lt);
                __syncwarp();
                if (b >= 0) {
                    if (perm) perm[slot] = (int32_t)i;
                    if (lane == __ffs(peers) - 1) run[b] += __popc(peers);
                }
                if (rank && i < c1) rank[i] = b >= 0 ? (int32_t)slot : -1;
                __syncwarp();
            }
        }
    }
}

// dst[rank[r]] = src[r] for rows of `words` units of U (rows with rank < 0 are skipped).  The
// reads stream through src in order; the writes of one block land close together in time,
// so partly written sectors merge in L2.
template <typename U>
__global__ void __launch_bounds__(256) k_scatter_rows(const U* __restrict__ src, U* __restrict__ dst, long long words,
                                                      const int32_t* __restrict__ rank, long long n_rows)
{
    const long long total = n_rows * words;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / words, w = t - r * words;
        const int32_t d = __ldg(rank + r);
        if (d >= 0) dst[(long long)d * words + w] = __ldg(src + t);
    }
}

// dst[r] = src[perm[r]] for rows of `words` units of U.
template <typename U>
__global__ void __launch_bounds__(256) k_gather_rows(const U* __restrict__ src, U* __restrict__ dst, long long words,
                                                     const int32_t* __restrict__ perm, long long n_rows)
{
    const long long total = n_rows * words;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / words, w = t - r * words;
        dst[t] = __ldg(src + (long long)__ldg(perm + r) * words + w);
    }
}

static bool make_params(const float* pmin, const float* pmax, const int32_t* grid, PartParams* P)
{
    if (!pmin || !pmax || !grid) return false;
    long long nb = 1;
    for (int a = 0; a < 3; a++) {
        if (grid[a] < 1 || grid[a] > CGS_PARTITION_MAX_CELLS) return false;
        if (!(std::isfinite(pmin[a]) && std::isfinite(pmax[a]) && pmax[a] > pmin[a])) return false;
        nb *= grid[a];
        P->pmin[a] = pmin[a];
        P->pmax[a] = pmax[a];
        P->g[a] = grid[a];
        for (int i = 0; i <= CGS_PARTITION_MAX_CELLS; i++) {
            // b_i = 4 i / g - 2, each operation rounded to FP32 (host SSE arithmetic)
            volatile float q = (4.0f * (float)i) / (float)grid[a];
            P->bnd[a][i] = (i >= 1 && i < grid[a]) ? (float)(q - 2.0f) : 0.0f;
        }
    }
    if (nb > CGS_PARTITION_MAX_BLOCKS) return false;
    P->nb = (int)nb;
    return true;
}

struct PartPlan {
    long long ch, n_chunks, counts;
};

static PartPlan plan(long long n, int nb)
{
    PartPlan p;
    long long ch = (n * nb + PART_MAX_COUNTS - 1) / PART_MAX_COUNTS;
    ch = ((ch + 31) / 32) * 32;
    p.ch = ch < PART_MIN_CHUNK ? PART_MIN_CHUNK : ch;
    p.n_chunks = n > 0 ? (n + p.ch - 1) / p.ch : 1;
    p.counts = p.n_chunks * nb;
    return p;
}

static size_t part_ws_bytes(const PartPlan& p, size_t* off_cnt, size_t* off_lb)
{
    const size_t hdr = (sizeof(Header) + 255) & ~(size_t)255;
    const size_t cnt = (((size_t)p.counts * 4) + 255) & ~(size_t)255;
    const size_t lb = (((size_t)((p.counts + SCAN_TILE - 1) / SCAN_TILE) * 8) + 255) & ~(size_t)255;
    if (off_cnt) *off_cnt = hdr;
    if (off_lb) *off_lb = hdr + cnt;
    return hdr + cnt + lb;
}

static bool valid_rows(const float* d_pos, int64_t n, int64_t stride)
{
    return n >= 0 && n < (1ll << 31) && stride >= 3 && (n == 0 || d_pos);
}

}  // namespace cgs

using namespace cgs;

extern "C" int32_t cgs_contract(const float* d_pos, int64_t n, int64_t stride, const float* pmin, const float* pmax,
                                float* d_out, void* stream)
{
    PartParams P;
    const int32_t one[3] = {1, 1, 1};
    if (!valid_rows(d_pos, n, stride) || (n > 0 && !d_out) || !make_params(pmin, pmax, one, &P))
        return CGS_ERR_INVALID_ARGUMENT;
    if (n == 0) return CGS_OK;
    const long long grid = std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 8);
    k_contract<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(P, d_pos, stride, n, d_out);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

extern "C" int32_t cgs_pose_blocks(const float* d_pos, int64_t n, int64_t stride, const float* pmin,
                                   const float* pmax, const int32_t* grid, int32_t* d_block, void* stream)
{
    PartParams P;
    if (!valid_rows(d_pos, n, stride) || (n > 0 && !d_block) || !make_params(pmin, pmax, grid, &P))
        return CGS_ERR_INVALID_ARGUMENT;
    if (n == 0) return CGS_OK;
    const long long g = std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 8);
    k_point_blocks<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(P, d_pos, stride, n, d_block);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

extern "C" int64_t cgs_partition_workspace_bytes(int64_t n, const int32_t* grid)
{
    if (n < 0 || n >= (1ll << 31) || !grid) return -1;
    long long nb = 1;
    for (int a = 0; a < 3; a++) {
        if (grid[a] < 1 || grid[a] > CGS_PARTITION_MAX_CELLS) return -1;
        nb *= grid[a];
    }
    if (nb > CGS_PARTITION_MAX_BLOCKS) return -1;
    return (int64_t)part_ws_bytes(plan(n, (int)nb), nullptr, nullptr);
}

extern "C" int32_t cgs_partition(const float* d_pos, int64_t n, int64_t stride, const float* pmin, const float* pmax,
                                 const int32_t* grid, int32_t* d_block, int64_t* d_block_offset, int32_t* d_perm,
                                 int32_t* d_rank, void* d_ws, int64_t ws_bytes, void* stream)
{
    PartParams P;
    if (!valid_rows(d_pos, n, stride) || !d_block_offset || (n > 0 && !d_block) || !make_params(pmin, pmax, grid, &P))
        return CGS_ERR_INVALID_ARGUMENT;
    const PartPlan pl = plan(n, P.nb);
    size_t off_cnt = 0, off_lb = 0;
    const size_t need = part_ws_bytes(pl, &off_cnt, &off_lb);
    if (!d_ws || ws_bytes < (int64_t)need) return CGS_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = static_cast<char*>(d_ws);
    Header* hdr = reinterpret_cast<Header*>(ws);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(ws + off_cnt);
    unsigned long long* lb = reinterpret_cast<unsigned long long*>(ws + off_lb);
    // header (status, scan tile counter) and look-back words start cleared
    if (cudaMemsetAsync(hdr, 0, sizeof(Header), st) != cudaSuccess) return CGS_ERR_CUDA;
    if (cudaMemsetAsync(lb, 0, need - off_lb, st) != cudaSuccess) return CGS_ERR_CUDA;
    const int n_sm = device_sm_count();
    const size_t smem = (size_t)PART_WARPS * P.nb * sizeof(uint32_t);
    const long long warps_needed = pl.n_chunks;
    const long long ctas = std::max<long long>(1, std::min<long long>((warps_needed + PART_WARPS - 1) / PART_WARPS,
                                                                      (long long)n_sm * 4));
    if (n > 0) {
        k_part_assign<<<(unsigned)ctas, PART_THREADS, smem, st>>>(P, d_pos, stride, n, pl.ch, pl.n_chunks, d_block,
                                                                  cnt);
    } else {
        if (cudaMemsetAsync(cnt, 0, (size_t)pl.counts * 4, st) != cudaSuccess) return CGS_ERR_CUDA;
    }
    PartScanOp op{cnt, pl.n_chunks, pl.counts, d_block_offset};
    const long long scan_ctas = std::max<long long>(1, std::min<long long>((pl.counts + SCAN_TILE - 1) / SCAN_TILE,
                                                                           (long long)n_sm * 8));
    k_scan<PartScanOp><<<(unsigned)scan_ctas, SCAN_THREADS, 0, st>>>(op, lb, hdr->ctr + 0, hdr);
    int launched = (n > 0 ? 1 : 0) + 1;
    if ((d_perm || d_rank) && n > 0) {
        k_part_scatter<<<(unsigned)ctas, PART_THREADS, smem, st>>>(P.nb, n, pl.ch, pl.n_chunks, d_block, cnt, d_perm,
                                                                   d_rank);
        launched++;
    }
    count_launches(launched);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

extern "C" int32_t cgs_partition_status(const void* d_ws, void* stream)
{
    if (!d_ws) return CGS_ERR_INVALID_ARGUMENT;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CGS_ERR_CUDA;
    Header h;
    if (cudaMemcpy(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return CGS_ERR_CUDA;
    return (h.status & ST_SPIN) ? CGS_ERR_SPIN_TIMEOUT : CGS_OK;
}

extern "C" int32_t cgs_scatter_rows(const void* d_src, void* d_dst, int64_t row_bytes, const int32_t* d_rank,
                                    int64_t n_rows, void* stream)
{
    if (n_rows < 0 || row_bytes <= 0 || row_bytes % 4 != 0) return CGS_ERR_INVALID_ARGUMENT;
    if (n_rows == 0) return CGS_OK;
    if (!d_src || !d_dst || !d_rank) return CGS_ERR_INVALID_ARGUMENT;
    const uintptr_t al = (uintptr_t)d_src | (uintptr_t)d_dst | (uintptr_t)row_bytes;
    const int unit = (al % 16 == 0) ? 16 : ((al % 8 == 0) ? 8 : 4);
    const long long words = row_bytes / unit;
    const long long total = n_rows * words;
    const long long g = std::max<long long>(1, std::min<long long>((total + 255) / 256, (long long)device_sm_count() * 16));
    cudaStream_t st = (cudaStream_t)stream;
    if (unit == 16)
        k_scatter_rows<uint4><<<(unsigned)g, 256, 0, st>>>((const uint4*)d_src, (uint4*)d_dst, words, d_rank, n_rows);
    else if (unit == 8)
        k_scatter_rows<uint2><<<(unsigned)g, 256, 0, st>>>((const uint2*)d_src, (uint2*)d_dst, words, d_rank, n_rows);
    else
        k_scatter_rows<uint32_t><<<(unsigned)g, 256, 0, st>>>((const uint32_t*)d_src, (uint32_t*)d_dst, words, d_rank,
                                                             n_rows);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}

extern "C" int32_t cgs_gather_rows(const void* d_src, void* d_dst, int64_t row_bytes, const int32_t* d_perm,
                                   int64_t n_rows, void* stream)
{
    if (n_rows < 0 || row_bytes <= 0 || row_bytes % 4 != 0) return CGS_ERR_INVALID_ARGUMENT;
    if (n_rows == 0) return CGS_OK;
    if (!d_src || !d_dst || !d_perm) return CGS_ERR_INVALID_ARGUMENT;
    const uintptr_t al = (uintptr_t)d_src | (uintptr_t)d_dst | (uintptr_t)row_bytes;
    const int unit = (al % 16 == 0) ? 16 : ((al % 8 == 0) ? 8 : 4);
    const long long words = row_bytes / unit;
    const long long total = n_rows * words;
    const long long g = std::max<long long>(1, std::min<long long>((total + 255) / 256, (long long)device_sm_count() * 16));
    cudaStream_t st = (cudaStream_t)stream;
    if (unit == 16)
        k_gather_rows<uint4><<<(unsigned)g, 256, 0, st>>>((const uint4*)d_src, (uint4*)d_dst, words, d_perm, n_rows);
    else if (unit == 8)
        k_gather_rows<uint2><<<(unsigned)g, 256, 0, st>>>((const uint2*)d_src, (uint2*)d_dst, words, d_perm, n_rows);
    else
        k_gather_rows<uint32_t><<<(unsigned)g, 256, 0, st>>>((const uint32_t*)d_src, (uint32_t*)d_dst, words, d_perm,
                                                            n_rows);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? CGS_OK : CGS_ERR_CUDA;
}
