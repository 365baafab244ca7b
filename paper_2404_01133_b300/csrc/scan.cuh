// Single-pass exclusive scan of a u32 sequence with a per-item action (decoupled look-back,
// u64 running totals).  Shared by the tile-list stage and the block partition.
#pragma once

#include "common.cuh"

namespace cgs {

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

}  // namespace cgs
