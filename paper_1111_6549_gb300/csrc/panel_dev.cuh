// panel_dev.cuh -- the pivot search of one 64-column stripe as device
// functions, shared by the stripe kernel (one matrix) and the batched kernel
// (one matrix per CTA).  Algorithm 1's column-wise search: leftmost column
// with a nonzero among the remaining rows, first such row in the current
// order, rows exchanged by swaps.
#pragma once

#include "common.cuh"

#include <climits>

namespace gf2 {

// Transpose a 32 x 32 bit block held one row per lane (bit c of lane r =
// entry (r, c)) so that lane c receives column c (bit r = entry (r, c)):
// five rounds of swapping the off-diagonal sub-blocks of size 16, 8, 4, 2, 1.
__device__ __forceinline__ unsigned transpose32(unsigned x)
{
    const int lane = threadIdx.x & 31;
    const unsigned masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int j = 16 >> k;
        const unsigned m = masks[k];
        const unsigned y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? (((y >> j) & m) | (x & ~m)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

// Shared state of one stripe's pivot search.
struct PanelShared {
    uint64_t E[KS], L[KS];     // pivot rows' stripe words (echelon) and L coefficients
    int32_t t[KS];             // window slot where pivot p was found (swap partner)
    uint8_t j[KS];             // pivot column offsets
    int32_t perm[PANEL_WIN];   // window slot -> original slot of its content
    int32_t Soff[SMAX];        // staged rows: position offsets
    int64_t Ssrc[SMAX];        //              physical source rows
    int fail, rbar, nS, maxpos, best;
    unsigned long long colmask;
    // block-wide path: compaction counts, and the rows with a zero stripe
    // word that swaps moved (current position offset, source offset)
    int cnt, nz;
    int wcnt[32];
    int32_t zpos[KS], zsrc[KS];
};

// Fast path, called by one whole warp: a bit-sliced window of up to 128 rows
// (lane l owns columns l and l+32 as 128-row masks).  Sets sh.fail when some
// column's pivot may lie outside the window; otherwise sh.rbar, E, L, t, j
// and the staged-row list.
__device__ __forceinline__ void panel_window(const uint64_t *__restrict__ A, int64_t r, int64_t ld,
                                             int64_t cw, int64_t rows, int keff, PanelShared &sh)
{
    const int lane = threadIdx.x & 31;
        const int Wn = (int)min(rows, (int64_t)PANEL_WIN);
        // load: lane l holds window rows l, l+32, l+64, l+96 ...
        uint64_t rw[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int sl = b * 32 + lane;
            rw[b] = (sl < Wn) ? A[(r + sl) * ld + cw] : 0ull;
        }
        // ... transposed so that lane l owns columns l and l+32 as 128-row masks
        uint64_t c0lo, c0hi, c1lo, c1hi;
        {
            unsigned t0[4], t1[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                t0[b] = transpose32((unsigned)rw[b]);
                t1[b] = transpose32((unsigned)(rw[b] >> 32));
            }
            c0lo = ((uint64_t)t0[1] << 32) | t0[0];
            c0hi = ((uint64_t)t0[3] << 32) | t0[2];
            c1lo = ((uint64_t)t1[1] << 32) | t1[0];
            c1hi = ((uint64_t)t1[3] << 32) | t1[2];
        }
        for (int x = lane; x < PANEL_WIN; x += 32) sh.perm[x] = x;
        __syncwarp();
        // L columns (pivot p's column = rows eliminated by it), lane owns p = lane, lane + 32
        uint64_t l0lo = 0, l0hi = 0, l1lo = 0, l1hi = 0;
        int p = 0, tmax = -1;
        bool fail = false;
        for (int j = 0; j < keff && p < Wn; ++j) {
            const int owner = j & 31;
            uint64_t jlo = __shfl_sync(0xffffffffu, (j < 32) ? c0lo : c1lo, owner);
            uint64_t jhi = __shfl_sync(0xffffffffu, (j < 32) ? c0hi : c1hi, owner);
            const uint64_t ge_lo = (p < 64) ? (~0ull << p) : 0ull;
            const uint64_t ge_hi = (p < 64) ? ~0ull : (~0ull << (p - 64));
            const uint64_t clo = jlo & ge_lo, chi = jhi & ge_hi;
            int t;
            if (clo) t = __ffsll((long long)clo) - 1;
            else if (chi) t = 64 + __ffsll((long long)chi) - 1;
            else {
                if (Wn < rows) { fail = true; break; }   // the pivot may lie outside the window
                continue;                                // column j has no pivot
            }
            // exchange rows p and t in every 128-row mask
            const uint64_t mp_lo = (p < 64) ? (1ull << p) : 0ull, mp_hi = (p < 64) ? 0ull : (1ull << (p - 64));
            const uint64_t mt_lo = (t < 64) ? (1ull << t) : 0ull, mt_hi = (t < 64) ? 0ull : (1ull << (t - 64));
            const uint64_t both_lo = mp_lo | mt_lo, both_hi = mp_hi | mt_hi;
#define GF2_SWAPROWS(lo, hi)                                                        \
            do {                                                                    \
                const bool d_ = (((lo) & mp_lo) | ((hi) & mp_hi)) != 0ull;          \
                const bool e_ = (((lo) & mt_lo) | ((hi) & mt_hi)) != 0ull;          \
                if (d_ != e_) { (lo) ^= both_lo; (hi) ^= both_hi; }                 \
            } while (0)
            GF2_SWAPROWS(jlo, jhi);
            const uint64_t gt_lo = (p >= 63) ? 0ull : (~0ull << (p + 1));
            const uint64_t gt_hi = (p < 63) ? ~0ull : ((p - 63) >= 64 ? 0ull : (~0ull << (p - 63)));
            const uint64_t rlo = jlo & gt_lo, rhi = jhi & gt_hi;   // rows below p holding column j
            GF2_SWAPROWS(c0lo, c0hi);
            GF2_SWAPROWS(c1lo, c1hi);
            GF2_SWAPROWS(l0lo, l0hi);
            GF2_SWAPROWS(l1lo, l1hi);
#undef GF2_SWAPROWS
            // the pivot row's entry in each owned column decides whether it is added
            if (((c0lo & mp_lo) | (c0hi & mp_hi)) != 0ull) { c0lo ^= rlo; c0hi ^= rhi; }
            if (((c1lo & mp_lo) | (c1hi & mp_hi)) != 0ull) { c1lo ^= rlo; c1hi ^= rhi; }
            if (lane == (p & 31)) {
                if (p < 32) { l0lo = rlo; l0hi = rhi; } else { l1lo = rlo; l1hi = rhi; }
            }
            if (lane == 0) {
                sh.t[p] = t;
                sh.j[p] = (uint8_t)j;
                const int a = sh.perm[p];
                sh.perm[p] = sh.perm[t];
                sh.perm[t] = a;
            }
            tmax = max(tmax, t);
            ++p;
        }
        if (!fail) {
            // rows 0..p-1 of the window now hold the pivots: transpose the column
            // masks back into rows (lane r gets rows r and r + 32)
            {
                const unsigned e00 = transpose32((unsigned)c0lo), e01 = transpose32((unsigned)c1lo);
                const unsigned e10 = transpose32((unsigned)(c0lo >> 32)), e11 = transpose32((unsigned)(c1lo >> 32));
                const unsigned f00 = transpose32((unsigned)l0lo), f01 = transpose32((unsigned)l1lo);
                const unsigned f10 = transpose32((unsigned)(l0lo >> 32)), f11 = transpose32((unsigned)(l1lo >> 32));
                const int q0 = lane, q1 = lane + 32;
                if (q0 < p) {
                    sh.E[q0] = ((uint64_t)e01 << 32) | e00;
                    sh.L[q0] = ((((uint64_t)f01 << 32) | f00)) & ((q0 == 0) ? 0ull : (~0ull >> (64 - q0)));
                }
                if (q1 < p) {
                    sh.E[q1] = ((uint64_t)e11 << 32) | e10;
                    sh.L[q1] = ((((uint64_t)f11 << 32) | f10)) & (~0ull >> (64 - q1));
                }
            }
            __syncwarp();
            // staged rows: pivot rows first, then rows displaced into [p, tmax]
            for (int k = lane; k < p; k += 32) { sh.Soff[k] = k; sh.Ssrc[k] = r + sh.perm[k]; }
            int base = p;
            for (int b0 = p; b0 <= tmax; b0 += 32) {
                const int sl = b0 + lane;
                const bool mv = sl <= tmax && sh.perm[sl] != sl;
                const unsigned bm = __ballot_sync(0xffffffffu, mv);
                if (mv) {
                    const int k = base + __popc(bm & ((1u << lane) - 1u));
                    sh.Soff[k] = sl;
                    sh.Ssrc[k] = r + sh.perm[sl];
                }
                base += __popc(bm);
            }
            if (lane == 0) { sh.nS = base; sh.maxpos = max(p - 1, tmax); }
        }
        if (lane == 0) { sh.fail = fail ? 1 : 0; sh.rbar = p; }
    }

// Block-wide path (every thread of the block): Algorithm 1's search over all
// remaining rows.  Rows whose stripe word is zero can never hold a pivot and
// are never changed by the stripe's eliminations, so only the nonzero rows
// are gathered (a stable, position-ordered compaction into the scratch) and
// searched; a zero row matters only when a swap moves it, and the few such
// moves are tracked in shared memory.  Sparse stripes (the regime of Section
// 4's Figure) thus cost time in proportion to their nonzero rows.  Columns
// that are zero in every remaining row are skipped outright.
__device__ __forceinline__ void panel_block(const uint64_t *__restrict__ A, int64_t r, int64_t ld,
                                            int64_t cw, int64_t rows, int keff, PanelScratch gs,
                                            PanelShared &sh, int32_t *fallbacks)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;
    if (tid == 0) {
        sh.colmask = 0;
        sh.cnt = 0;
        sh.nz = 0;
        if (fallbacks) atomicAdd(fallbacks, 1);
    }
    __syncthreads();
    // 1. stable compaction of the rows with a nonzero stripe word: each
    // thread counts a contiguous chunk of rows, a block-wide exclusive scan of
    // the counts gives every chunk its output offset, a second pass writes
    unsigned long long orv = 0;
    const int64_t chunk = (rows + nthr - 1) / nthr;
    const int64_t c0 = min(rows, (int64_t)tid * chunk), c1 = min(rows, c0 + chunk);
    int mine = 0;
    for (int64_t sl = c0; sl < c1; ++sl) {
        const uint64_t v = A[(r + sl) * ld + cw];
        orv |= v;
        mine += (v != 0ull);
    }
    int incl = mine;                              // inclusive scan inside the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) sh.wcnt[warp] = incl;
    __syncthreads();
    int off = incl - mine;
    for (int w2 = 0; w2 < warp; ++w2) off += sh.wcnt[w2];
    if (tid == nthr - 1) sh.cnt = off + mine;
    for (int64_t sl = c0; sl < c1; ++sl) {
        const uint64_t v = A[(r + sl) * ld + cw];
        if (v != 0ull) {
            gs.val[off] = v;
            gs.lb[off] = 0;
            gs.src[off] = (int32_t)sl;
            gs.pos[off] = (int32_t)sl;
            ++off;
        }
    }
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)orv);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(orv >> 32));
    if (lane == 0) atomicOr(&sh.colmask, ((unsigned long long)hi << 32) | lo);
    __syncthreads();
    const uint64_t colmask = sh.colmask;
    const int K = sh.cnt;
    // 2. column-wise search and eager elimination over the gathered rows
    int p = 0, first = 0;                         // pivots so far; first entry not yet retired
    for (int j = 0; j < keff && first < K; ++j) {
        if (!((colmask >> j) & 1ull)) continue;
        if (tid == 0) sh.best = INT_MAX;
        __syncthreads();
        for (int base = first; base < K; base += nthr) {
            const int k = base + tid;
            const bool hit = k < K && gs.pos[k] >= 0 && ((gs.val[k] >> j) & 1ull);
            if (__syncthreads_or(hit)) {
                if (hit) atomicMin(&sh.best, k);
                __syncthreads();
                break;
            }
        }
        const int kt = sh.best;
        __syncthreads();                              // everyone has kt before sh.best is reused
        if (kt == INT_MAX) continue;
        if (tid == 0) {
            // the pivot row (entry kt, at position t) swaps with the row at
            // position p: entry `first` if it sits there, else a zero row
            const int t = gs.pos[kt];
            const uint64_t tv = gs.val[kt], tl = gs.lb[kt];
            const int32_t ts = gs.src[kt];
            sh.t[p] = t;
            sh.j[p] = (uint8_t)j;
            sh.E[p] = tv;
            sh.L[p] = tl;
            sh.Soff[p] = p;
            sh.Ssrc[p] = r + ts;
            if (gs.pos[first] == p) {
                // first (the row at p) takes the pivot's place at t; the pivot retires
                if (kt != first) {
                    gs.val[kt] = gs.val[first];
                    gs.lb[kt] = gs.lb[first];
                    gs.src[kt] = gs.src[first];
                }
                gs.pos[first] = -1;
            } else {
                // a zero row sits at p: it moves to t
                int z = -1;
                for (int q = 0; q < sh.nz; ++q)
                    if (sh.zpos[q] == p) z = q;
                if (z < 0) {
                    z = sh.nz++;
                    sh.zsrc[z] = p;
                }
                sh.zpos[z] = t;
                gs.pos[kt] = -1;
            }
            int f = first;
            while (f < K && gs.pos[f] < 0) ++f;
            sh.best = f;                              // the new first live entry
        }
        __syncthreads();
        first = sh.best;
        const uint64_t pv = sh.E[p];
        const uint64_t bitp = 1ull << p;
        for (int k = first + tid; k < K; k += nthr) {
            const uint64_t v = gs.val[k];
            if (gs.pos[k] >= 0 && ((v >> j) & 1ull)) {
                gs.val[k] = v ^ pv;
                gs.lb[k] |= bitp;
            }
        }
        ++p;
        __syncthreads();
    }
    // 3. staged rows: the pivots, then every row a swap moved
    if (tid == 0) sh.nS = p;
    __syncthreads();
    for (int k = first + tid; k < K; k += nthr) {
        const int32_t ps = gs.pos[k];
        if (ps >= 0 && ps != gs.src[k]) {
            const int q = atomicAdd(&sh.nS, 1);
            sh.Soff[q] = ps;
            sh.Ssrc[q] = r + gs.src[k];
        }
    }
    if (tid < sh.nz && sh.zpos[tid] != sh.zsrc[tid]) {
        const int q = atomicAdd(&sh.nS, 1);
        sh.Soff[q] = sh.zpos[tid];
        sh.Ssrc[q] = r + sh.zsrc[tid];
    }
    __syncthreads();
    if (tid == 0) {
        int mx = p - 1;
        for (int q = 0; q < sh.nS; ++q) mx = max(mx, (int)sh.Soff[q]);
        sh.rbar = p;
        sh.maxpos = mx;
    }
    __syncthreads();
}

// Rows of L11^-1 (L11 unit lower triangular, rows Lrows[0..rbar)), by one
// warp: forward substitution per column (lane owns columns lane and
// lane + 32), rows collected by ballot; lane 0 writes out[p].
__device__ __forceinline__ void warp_lower_inverse(const uint64_t *Lrows, int rbar, uint64_t *out)
{
    const int lane = threadIdx.x & 31;
    uint64_t x0 = 0, x1 = 0;
    for (int p = 0; p < rbar; ++p) {
        const uint64_t Lp = Lrows[p];
        x0 |= (uint64_t)((((p == lane) ? 1 : 0) ^ __popcll(Lp & x0)) & 1) << p;
        x1 |= (uint64_t)((((p == lane + 32) ? 1 : 0) ^ __popcll(Lp & x1)) & 1) << p;
    }
    for (int p = 0; p < rbar; ++p) {
        const unsigned lo = __ballot_sync(0xffffffffu, (x0 >> p) & 1ull);
        const unsigned hi = __ballot_sync(0xffffffffu, (x1 >> p) & 1ull);
        if (lane == 0) out[p] = ((uint64_t)hi << 32) | lo;
    }
}

}  // namespace gf2
