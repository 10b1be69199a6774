// tables_dev.cuh -- the shared-memory table build of the tabulated update
// (Algorithm 6, MakeTable), used by both forms of the update kernel.
//
// Eight tables per 64-column stripe, table t holding all 256 combinations of
// generator rows 8t .. 8t+7 for one column tile of TW words.  Two tables share
// one 128-byte line (table 2a in bytes 0..63, table 2a+1 in bytes 64..127).
#pragma once

#include "common.cuh"

namespace gf2 {

// 512 threads: table tau (8) x segment q of 32 entries (8) x word w (8).
// Entries are built by doubling inside 32-entry Gray-code segments (255
// additions per table and word, the count of Algorithm 6).
__device__ __forceinline__ void build_tables(uint64_t *T, const uint64_t *const *gen, int64_t wbase,
                                             int64_t W)
{
    const int t = threadIdx.x;
    const int w = t & 7, q = (t >> 3) & 7, tau = t >> 6;
    const int64_t word = wbase + w;
    const bool inr = word < W;
    uint64_t g[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint64_t *p = gen[8 * tau + b];
        g[b] = (p != nullptr && inr) ? p[word] : 0ull;
    }
    uint64_t val = ((q & 1) ? g[5] : 0ull) ^ ((q & 2) ? g[6] : 0ull) ^ ((q & 4) ? g[7] : 0ull);
    uint64_t *Tt = T + (tau >> 1) * (256 * TAB_LINE) + (tau & 1) * TW + w;
    int x = 0;
    Tt[(32 * q) * TAB_LINE] = val;
#pragma unroll
    for (int i = 1; i < 32; ++i) {
        // Gray code: step i flips bit b = number of trailing zeros of i
        const int b = (i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : 4;
        x ^= 1 << b;
        val ^= g[b];
        Tt[(32 * q + x) * TAB_LINE] = val;
    }
}

// Wide form: 128-byte tiles (WT words), table t < 8 holding the 128
// combinations of generator rows 7t .. 7t+6, table 8 the 256 combinations of
// rows 56 .. 63; only the words [w_lo, W) of the tile are built.  Work items are (32-entry segment, word): 8 x 4 + 8 = 40
// segments x 16 words = 640 items over the block's threads; each item walks
// its segment in Gray-code order (31 additions after the segment's base).
__device__ __forceinline__ void build_wide_tables(uint64_t *T, const uint64_t *const *gen, int64_t wbase,
                                                  int64_t W, int64_t w_lo = 0)
{
    for (int item = threadIdx.x; item < 40 * WT; item += blockDim.x) {
        const int w = item % WT, seg = item / WT;
        // words outside [w_lo, W) are never stored back: their entries may stay stale
        if (wbase + w < w_lo || wbase + w >= W) continue;
        const int t = seg < 32 ? seg >> 2 : 8;       // table
        const int q = seg < 32 ? seg & 3 : seg - 32; // segment: index bits 5.. of the table
        const int nb = t < 8 ? 7 : 8;                // index bits of the table
        const int64_t word = wbase + w;
        const bool inr = word < W;
        uint64_t g[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint64_t *p = b < nb ? gen[7 * t + b] : nullptr;
            g[b] = (p != nullptr && inr) ? p[word] : 0ull;
        }
        uint64_t val = ((q & 1) ? g[5] : 0ull) ^ ((q & 2) ? g[6] : 0ull) ^ ((q & 4) ? g[7] : 0ull);
        uint64_t *Tt = T + (int64_t)(128 * t + 32 * q) * WT + w;
        int x = 0;
        Tt[0] = val;
#pragma unroll
        for (int i = 1; i < 32; ++i) {
            const int b = (i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : 4;
            x ^= 1 << b;
            val ^= g[b];
            Tt[x * WT] = val;
        }
    }
}

// As build_wide_tables, with the 64 generator rows of the tile in shared
// memory (G[row * WT + word]).
__device__ __forceinline__ void build_wide_tables_smem(uint64_t *T, const uint64_t *G)
{
    for (int item = threadIdx.x; item < 40 * WT; item += blockDim.x) {
        const int w = item % WT, seg = item / WT;
        const int t = seg < 32 ? seg >> 2 : 8;
        const int q = seg < 32 ? seg & 3 : seg - 32;
        const int nb = t < 8 ? 7 : 8;
        uint64_t g[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) g[b] = b < nb ? G[(7 * t + b) * WT + w] : 0ull;
        uint64_t val = ((q & 1) ? g[5] : 0ull) ^ ((q & 2) ? g[6] : 0ull) ^ ((q & 4) ? g[7] : 0ull);
        uint64_t *Tt = T + (int64_t)(128 * t + 32 * q) * WT + w;
        int x = 0;
        Tt[0] = val;
#pragma unroll
        for (int i = 1; i < 32; ++i) {
            const int b = (i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : 4;
            x ^= 1 << b;
            val ^= g[b];
            Tt[x * WT] = val;
        }
    }
}

}  // namespace gf2
