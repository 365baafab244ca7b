// Shared definitions of libcgs: frame workspace layout, device status, small helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cgs.h"

namespace cgs {

// ---------------------------------------------------------------------------------------
// device status and counters (first bytes of every frame workspace; zeroed per forward)
// ---------------------------------------------------------------------------------------
enum : uint32_t { ST_CAPACITY = 1u << 0, ST_SPIN = 1u << 1, ST_UNSUPPORTED = 1u << 2 };

// Dynamic work counters of the single-pass (decoupled look-back) and persistent kernels.
enum { CTR_SCAN_RANGES = 2, CTR_BIG = 3, CTR_SELECT = 5, N_CTR = 8 };

struct Header {
    uint32_t status;
    uint32_t n_sel;        // selected Gaussians summed over views, capped at n_cap
    uint32_t n_vis;        // visible (tiles touched > 0)
    uint32_t reserved;
    unsigned long long n_sel_raw;
    unsigned long long k_total;
    unsigned long long pairs_fwd;
    unsigned long long pairs_bwd;
    unsigned long long steps_fwd;     // forward (warp, entry) steps visited
    unsigned long long steps_useful;  // of those, steps where an entry blended into a warp pixel
    uint32_t spin_giveups;
    uint32_t n_big;        // tiles too long for the ranking sort
    uint32_t ctr[N_CTR];
};

// A frame of at most TSUB_MAX_TILES (view, tile) pairs counts, ranges and scatters each tile's
// entries in TSUB sub-ranges (an entry's is the low bits of its selected index), so the
// scatter's cursors see a TSUB-th of a tile's entries each (the sub-ranges of a tile are
// contiguous and make up its range); larger frames, whose counters already spread over many
// tiles, keep one range per tile (Layout::tsub_sh).
constexpr int TSUB = 4;
constexpr long long TSUB_MAX_TILES = 65536;

// Polls of a look-back flag before a kernel gives up and latches ST_SPIN.
constexpr int SPIN_LIMIT = 1 << 22;

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_IPT;

// Pointers into one frame workspace.  Built on the host by make_layout (api.cu).
struct Layout {
    Header* hdr;
    // zeroed at every forward (one memset from hdr over zero_bytes)
    unsigned long long* scan_lb; // [scan tiles of V*T] look-back words of the tile-range scan
    uint32_t* tcnt;              // [V * T][1 << tsub_sh] entries per tile and sub-range
    uint32_t* tcur;              // [V * T][1 << tsub_sh] scatter cursors
    uint32_t* sel_done;          // [V] CTAs of the view that finished the selection's first phase
    // not zeroed
    uint32_t* ranges;            // [V * T][2] [start, end) of every tile's entries
    uint32_t* ssub;              // [V * T][1 << tsub_sh] start of every sub-range
    int tsub_sh;                 // log2 of the sub-ranges per tile: 2 (TSUB) or 0
    uint32_t* view_base;         // [V + 1] exclusive prefix of per-view selected counts
    uint32_t* view_cnt;          // [V] selected count per view
    uint32_t* n_seg;             // [V]
    uint32_t* seg_base;          // [V][NB + 1]
    long long* seg_off;          // [V][NB]
    int32_t* seg_blk;            // [V][NB] block of each selected segment
    int lod_mode;                // CGS_LOD_BLOCK or CGS_LOD_POINT (point mode: per-Gaussian level test)
    float lod_d1, lod_d2;        // FP32 thresholds of the point mode
    int8_t* levels;              // [V][NB]
    float4* rec;                 // [n_cap][3] (u, v, o, ext_x) (A', B', C', ext_y) (r, g, b, t)
    uint2* rect;                 // [n_cap] (x0 | y0 << 16, x1 | y1 << 16), tile units, end exclusive
    uint32_t* tt;                // [n_cap] tiles touched
    uint32_t* gidx;              // [n_cap] scene index
    unsigned long long* pkey;    // [n_cap] view << 32 | depth bits
    uint32_t* vis;               // [n_cap] visible selected indices, ascending
    unsigned long long* eraw;    // [k_cap] tile << 32 | j per entry; later scratch of the long-tile sort
    unsigned long long* ekey;    // [k_cap] depth bits << 32 | j, scattered into tile ranges
    uint32_t* tval;              // [k_cap] selected index per entry, (tile, depth, index) order
    uint32_t* tkey;              // [k_cap] tile id per entry, same order
    uint32_t* big;               // [V * T] tiles for the long-tile sort
    float4* gs;                  // [n_cap][3] screen-space gradients (du dv dA dB | dC do dr dg | db - - -)
    uint32_t* hits;              // optional [scene n]: pixels blending each scene Gaussian (added to)
    uint32_t* cbits;             // per (tile, warp): bit p set when entry p blends into any of the warp's pixels
    long long cbits_words;
    size_t zero_bytes;           // bytes to clear from hdr
    int count_pairs;             // the compositing backward counts its contributing pairs
    long long n_cap, k_cap;
    int V, W, H, B, tiles_x, tiles_y, T, NB;
};

// The L1 photometric loss (Sec. 3.2.3) folded into the compositing backward: each pixel's
// dL/dimage = sign(img - target) / count comes from the rendered image and the target where the
// backward reads it, so no gradient image is written or read, and mean |img - target| is added
// to *loss (one atomic add per CTA).  inv = 1 / count as the FP32 quotient 1.0f / (float)count.
struct L1In {
    const float* img;  // rendered image [V][3][H][W]
    const void* tgt;   // target, same layout: float, or uint8_t channel t standing for t / 255
    float* loss;
    float inv;
    int u8;            // target element type: 1 = uint8_t, 0 = float
};

// ---------------------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) { return *(const volatile uint32_t*)p; }
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) { *(volatile uint32_t*)p = v; }
__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p)
{
    return *(const volatile unsigned long long*)p;
}
__device__ __forceinline__ void st_volatile64(unsigned long long* p, unsigned long long v)
{
    *(volatile unsigned long long*)p = v;
}

__device__ __forceinline__ void latch(Header* h, uint32_t bits) { atomicOr(&h->status, bits); }

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Block-wide exclusive scan over blockDim.x (<= 1024, multiple of 32) values; returns the
// exclusive prefix and writes the total to *total.  `warp_buf` holds >= 33 entries.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T* warp_buf, T* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_buf[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? warp_buf[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) warp_buf[lane] = wi - w;
        if (lane == nw - 1) warp_buf[32] = wi;
    }
    __syncthreads();
    T res = warp_buf[warp] + inc - x;
    *total = warp_buf[32];
    __syncthreads();
    return res;
}

// Tile entries kept: min(k_total, k_cap) (the projection drops the rest and latches
// ST_CAPACITY).
__device__ __forceinline__ long long entries_kept(const Layout& L)
{
    const unsigned long long t = L.hdr->k_total;
    return t < (unsigned long long)L.k_cap ? (long long)t : L.k_cap;
}

// host helpers defined in api.cu: the library-wide launch counter and the SM count of the
// current device
void count_launches(int n);
int device_sm_count();

}  // namespace cgs
