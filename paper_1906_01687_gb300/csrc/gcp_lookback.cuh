// Ordered compaction across blocks (decoupled look-back), for the stratified
// zeros of Alg. 2: the first q accepted candidates in candidate order are
// kept, so every tile of candidates needs the number accepted before it.
//
// Tiles are numbered in the order blocks take them from a counter (so a tile
// only waits on tiles whose blocks are already running or done).  Each tile
// has one 64-bit word: a flag in the top two bits (count published, or
// inclusive prefix published) and the value below.  A tile publishes its
// count, then reads the earlier tiles' words 32 at a time (one per lane of
// its block's first warp) until it meets a published prefix with every tile
// between that one and itself at least counted, and publishes its own
// inclusive prefix.
#pragma once

#include <cstdint>

namespace gcpk {

constexpr unsigned long long kTileCount = 1ull << 62;   // tile word: this tile's count is published
constexpr unsigned long long kTilePrefix = 2ull << 62;  // tile word: its inclusive prefix is published
constexpr unsigned long long kTileValue = (1ull << 62) - 1ull;
constexpr int kSpinLimit = 1 << 21;  // polls of a look-back window before giving up

// Called by all 32 lanes of one warp of the tile's block.  words: the tile
// words (zero between uses); total: this tile's count.  Sets excl to the
// count of all earlier tiles and returns true, or returns false after
// kSpinLimit polls without progress (the tile's prefix is then never
// published).
__device__ __forceinline__ bool tile_lookback(unsigned long long* words, int64_t tile, int64_t total,
                                              int64_t& excl)
{
    const int lane = threadIdx.x & 31;
    excl = 0;
    if (tile == 0) {
        if (lane == 0) atomicExch(words, kTilePrefix | static_cast<unsigned long long>(total));
        return true;
    }
    if (lane == 0) atomicExch(words + tile, kTileCount | static_cast<unsigned long long>(total));
    int64_t hi = tile - 1;  // the window is tiles hi, hi - 1, ..., hi - 31 (lane i: tile hi - i)
    int spins = 0;
    while (true) {
        const int64_t j = hi - lane;
        unsigned long long w = kTilePrefix | 0ull;  // before tile 0: an empty prefix
        if (j >= 0) w = *reinterpret_cast<volatile unsigned long long*>(words + j);
        const unsigned long long flag = w & ~kTileValue;
        const unsigned not_ready = __ballot_sync(0xFFFFFFFFu, flag == 0ull);
        const unsigned prefix = __ballot_sync(0xFFFFFFFFu, flag == kTilePrefix);
        const int nearest = prefix ? __ffs(prefix) - 1 : 32;  // lowest lane: the nearest tile
        const unsigned needed = nearest >= 31 ? 0xFFFFFFFFu : (2u << nearest) - 1u;
        if (not_ready & needed) {
            if (++spins > kSpinLimit) return false;
            continue;
        }
        int64_t v = (lane <= nearest && j >= 0) ? static_cast<int64_t>(w & kTileValue) : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
        excl += v;
        if (nearest < 32) break;
        hi -= 32;
    }
    if (lane == 0) atomicExch(words + tile, kTilePrefix | static_cast<unsigned long long>(excl + total));
    return true;
}

// Exclusive rank of this thread's flag among its block's flags (thread
// order) and the block's count, for blocks of whole warps up to 1024
// threads.  sh_warp: 32 ints of shared memory.  Contains __syncthreads.
__device__ __forceinline__ int block_flag_rank(bool flag, int* sh_warp, int& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, flag);
    if (lane == 0) sh_warp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < nw; ++w) {
        const int c = sh_warp[w];
        before += w < warp ? c : 0;
        all += c;
    }
    __syncthreads();  // sh_warp may be reused
    total = all;
    return before + __popc(bal & ((1u << lane) - 1u));
}

}  // namespace gcpk
