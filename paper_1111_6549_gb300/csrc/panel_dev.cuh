// panel_dev.cuh -- the pivot search of one 64-column stripe as device
// functions, shared by the stripe kernel (one matrix) and the batched kernel
// (one matrix per CTA).  Algorithm 1's column-wise search: leftmost column
// with a nonzero among the remaining rows, first such row in the current
// order, rows exchanged by swaps.
#pragma once

#include "common.cuh"

#include <climits>

namespace gf2 {

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

// Where a row's stripe word lives while the previous stripe's trailing
// update may still be running (the look-ahead of the block-iterative PLE):
// rows that the previous stripe's swaps moved are read from its staged
// copies, which already hold their updated word of this stripe; every other
// row is read in place.  map == nullptr: every row in place.
struct PrevStage {
    const int32_t *map;   // the previous stripe's row map (position -> stripe * 256 + staged slot)
    const uint64_t *S;    // its staged rows
    int64_t ldS;
    int64_t r;            // its first row position
    int maxpos;           // its largest staged position offset
    int stripe;           // its index
};

__device__ __forceinline__ uint64_t stripe_word(const uint64_t *__restrict__ A, int64_t ld, int64_t cw, int64_t p,
                                                const PrevStage &ps)
{
    if (ps.map && p >= ps.r && p - ps.r <= ps.maxpos) {
        const int mv = ps.map[p];
        if (mv >= 0 && (mv >> 8) == ps.stripe) return ps.S[(int64_t)(mv & 255) * ps.ldS + cw];
    }
    return A[p * ld + cw];
}

// One of four registers by a warp-uniform index (no local-memory array).
template <typename T>
__device__ __forceinline__ T pick4(const T (&v)[4], int b)
{
    return b == 0 ? v[0] : b == 1 ? v[1] : b == 2 ? v[2] : v[3];
}

// Fast path, called by one whole warp: a window of up to 128 rows held in
// registers, lane l owning the window slots l, l+32, l+64 and l+96 (their
// stripe words, their L coefficients -- bit q: eliminated by pivot q -- and
// the slot their content came from).  A pivot step is four ballots for the
// slots holding column j, a find-first-set for the pivot slot t, one
// broadcast of the pivot row (plus an exchange with slot p when t != p) and
// a conditional XOR per owned slot.  Sets sh.fail when some column's pivot
// may lie outside the window; otherwise sh.rbar, E, L, t, j and the
// staged-row list.
__device__ __forceinline__ void panel_window(const uint64_t *__restrict__ A, int64_t r, int64_t ld,
                                             int64_t cw, int64_t rows, int keff, PanelShared &sh,
                                             const PrevStage ps = PrevStage{nullptr, nullptr, 0, 0, -1, -1})
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int Wn = (int)min(rows, (int64_t)PANEL_WIN);
    uint64_t R[4], Lc[4];
    int org[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int sl = b * 32 + lane;
        R[b] = (sl < Wn) ? stripe_word(A, ld, cw, r + sl, ps) : 0ull;
        Lc[b] = 0ull;
        org[b] = sl;
    }
    int p = 0, tmax = -1;
    bool fail = false;
    for (int j = 0; j < keff && p < Wn; ++j) {
        // slots holding column j, from slot p on
        const unsigned m0 = __ballot_sync(FULL, (unsigned)(R[0] >> j) & 1u);
        const unsigned m1 = __ballot_sync(FULL, (unsigned)(R[1] >> j) & 1u);
        const unsigned m2 = __ballot_sync(FULL, (unsigned)(R[2] >> j) & 1u);
        const unsigned m3 = __ballot_sync(FULL, (unsigned)(R[3] >> j) & 1u);
        const uint64_t lo = (((uint64_t)m1 << 32) | m0) & ((p < 64) ? (~0ull << p) : 0ull);
        const uint64_t hi = (((uint64_t)m3 << 32) | m2) & ((p < 64) ? ~0ull : (~0ull << (p - 64)));
        int t;
        if (lo) t = __ffsll((long long)lo) - 1;
        else if (hi) t = 64 + __ffsll((long long)hi) - 1;
        else {
            if (Wn < rows) { fail = true; break; }   // the pivot may lie outside the window
            continue;                                // column j has no pivot
        }
        const int bt = t >> 5, lt = t & 31, bp = p >> 5, lp = p & 31;
        const uint64_t prow = __shfl_sync(FULL, pick4(R, bt), lt);
        if (t != p) {
            // exchange slots p and t: slot p takes the pivot row, slot t the old row p
            const uint64_t plc = __shfl_sync(FULL, pick4(Lc, bt), lt);
            const int orgt = __shfl_sync(FULL, pick4(org, bt), lt);
            const uint64_t rowp = __shfl_sync(FULL, pick4(R, bp), lp);
            const uint64_t lcp = __shfl_sync(FULL, pick4(Lc, bp), lp);
            const int orgp = __shfl_sync(FULL, pick4(org, bp), lp);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (b == bp && lane == lp) { R[b] = prow; Lc[b] = plc; org[b] = orgt; }
                if (b == bt && lane == lt) { R[b] = rowp; Lc[b] = lcp; org[b] = orgp; }
            }
        }
        // eliminate column j from the slots after t that hold it (slot t now
        // holds the old row p, zero in column j)
        const uint64_t elo = lo & ((t >= 63) ? 0ull : (~0ull << (t + 1)));
        const uint64_t ehi = hi & ((t < 63) ? ~0ull : ((t - 63) >= 64 ? 0ull : (~0ull << (t - 63))));
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint64_t e = (b < 2) ? elo : ehi;
            const uint64_t sel = 0ull - ((e >> ((32 * b + lane) & 63)) & 1ull);
            R[b] ^= prow & sel;
            Lc[b] |= (1ull << p) & sel;
        }
        if (lane == 0) {
            sh.t[p] = t;
            sh.j[p] = (uint8_t)j;
        }
        tmax = max(tmax, t);
        ++p;
    }
    if (!fail) {
        // slots 0 .. p-1 hold the pivot rows (echelon); their L bits are below their index
        if (lane < p) {
            sh.E[lane] = R[0];
            sh.L[lane] = Lc[0] & ((lane == 0) ? 0ull : (~0ull >> (64 - lane)));
        }
        if (lane + 32 < p) {
            sh.E[lane + 32] = R[1];
            sh.L[lane + 32] = Lc[1] & (~0ull >> (32 - lane));
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) sh.perm[32 * b + lane] = org[b];
        __syncwarp();
        // staged rows: pivot rows first, then rows displaced into [p, tmax]
        for (int k = lane; k < p; k += 32) { sh.Soff[k] = k; sh.Ssrc[k] = r + sh.perm[k]; }
        int base = p;
        for (int b0 = p; b0 <= tmax; b0 += 32) {
            const int sl = b0 + lane;
            const bool mv = sl <= tmax && sh.perm[sl] != sl;
            const unsigned bm = __ballot_sync(FULL, mv);
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
                                            PanelShared &sh, int32_t *fallbacks,
                                            const PrevStage ps = PrevStage{nullptr, nullptr, 0, 0, -1, -1})
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
        const uint64_t v = stripe_word(A, ld, cw, r + sl, ps);
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
        const uint64_t v = stripe_word(A, ld, cw, r + sl, ps);
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


// Fast path over four warps (threads 0..127 of the block, every one of them
// must call it): the same search as panel_window, with window slot i held by
// thread i (its stripe word, its L coefficients, the slot its content came
// from).  Per column: one ballot per warp, the four ballots and then the
// pivot row (and the row it swaps with) exchanged through shared memory
// between two 128-thread barriers, and one conditional XOR per thread.  The
// exchange buffers alternate between two halves by step parity, so a step's
// writes never meet the previous step's reads.  Sets sh.fail exactly when
// panel_window would.
__device__ __forceinline__ void panel_bar128() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

__device__ __forceinline__ void panel_window4(const uint64_t *__restrict__ A, int64_t r, int64_t ld,
                                              int64_t cw, int64_t rows, int keff, PanelShared &sh,
                                              const PrevStage &ps)
{
    __shared__ unsigned sb[2][4];
    __shared__ uint64_t sv[2][2], sl[2][2];
    __shared__ int so[2][2];
    const int slot = threadIdx.x, lane = slot & 31, w = slot >> 5;
    const unsigned FULL = 0xffffffffu;
    const int Wn = (int)min(rows, (int64_t)PANEL_WIN);
    uint64_t R = (slot < Wn) ? stripe_word(A, ld, cw, r + slot, ps) : 0ull;
    uint64_t Lc = 0;
    int org = slot;
    int p = 0, tmax = -1, ph = 0;
    bool fail = false;
    for (int j = 0; j < keff && p < Wn; ++j) {
        const unsigned b = __ballot_sync(FULL, (unsigned)(R >> j) & 1u);
        if (lane == 0) sb[ph][w] = b;
        panel_bar128();
        const uint64_t lo = (((uint64_t)sb[ph][1] << 32) | sb[ph][0]) & ((p < 64) ? (~0ull << p) : 0ull);
        const uint64_t hi = (((uint64_t)sb[ph][3] << 32) | sb[ph][2]) & ((p < 64) ? ~0ull : (~0ull << (p - 64)));
        int t;
        if (lo) t = __ffsll((long long)lo) - 1;
        else if (hi) t = 64 + __ffsll((long long)hi) - 1;
        else {
            if (Wn < rows) { fail = true; break; }   // the pivot may lie outside the window
            ph ^= 1;
            continue;                                // column j has no pivot
        }
        // the pivot row (slot t) and the row it exchanges with (slot p)
        if (slot == t) { sv[ph][0] = R; sl[ph][0] = Lc; so[ph][0] = org; }
        if (slot == p) { sv[ph][1] = R; sl[ph][1] = Lc; so[ph][1] = org; }
        panel_bar128();
        const uint64_t prow = sv[ph][0];
        if (t != p) {
            if (slot == p) { R = prow; Lc = sl[ph][0]; org = so[ph][0]; }
            else if (slot == t) { R = sv[ph][1]; Lc = sl[ph][1]; org = so[ph][1]; }
        }
        // eliminate column j from the slots after p holding it (slot t now
        // holds the old row p, zero in column j)
        if (slot > p && ((R >> j) & 1ull)) {
            R ^= prow;
            Lc |= 1ull << p;
        }
        if (slot == 0) {
            sh.t[p] = t;
            sh.j[p] = (uint8_t)j;
        }
        tmax = max(tmax, t);
        ++p;
        ph ^= 1;
    }
    if (!fail) {
        // slots 0 .. p-1 hold the pivot rows (echelon); their L bits are below their index
        if (slot < p) {
            sh.E[slot] = R;
            sh.L[slot] = Lc & ((slot == 0) ? 0ull : (~0ull >> (64 - slot)));
        }
        sh.perm[slot] = org;
        panel_bar128();
        if (w == 0) {
            // staged rows: pivot rows first, then rows displaced into [p, tmax]
            for (int k = lane; k < p; k += 32) { sh.Soff[k] = k; sh.Ssrc[k] = r + sh.perm[k]; }
            int base = p;
            for (int b0 = p; b0 <= tmax; b0 += 32) {
                const int sl2 = b0 + lane;
                const bool mv = sl2 <= tmax && sh.perm[sl2] != sl2;
                const unsigned bm = __ballot_sync(FULL, mv);
                if (mv) {
                    const int k = base + __popc(bm & ((1u << lane) - 1u));
                    sh.Soff[k] = sl2;
                    sh.Ssrc[k] = r + sh.perm[sl2];
                }
                base += __popc(bm);
            }
            if (lane == 0) { sh.nS = base; sh.maxpos = max(p - 1, tmax); }
        }
    }
    if (slot == 0) { sh.fail = fail ? 1 : 0; sh.rbar = p; }
}

// Inverse of a 64 x 64 unit lower triangular matrix by one warp, in 32 x 32
// blocks: with L = [L1 0; C L2], L^-1 = [L1^-1 0; L2^-1 C L1^-1  L2^-1].
// Lane l forms column l of L1^-1 and of L2^-1 by forward substitution (two
// independent 32-step chains), then column l of the lower-left block as
// L2^-1 (C (column l of L1^-1)) by parities; rows come out by ballot.
// Lrows[p] (p < n) holds row p's strictly lower bits (bits at or above the
// diagonal are ignored); rows p >= n count as identity rows.  Writes row p
// of L^-1 to out[p] (and out2[p]) for p < n.
__device__ __forceinline__ void warp_lower_inverse_blocked(const uint64_t *Lrows, int n, uint64_t *out,
                                                           uint64_t *out2 = nullptr)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    auto row = [&](int p) -> uint64_t { return p < n ? (Lrows[p] & ((1ull << p) - 1ull)) : 0ull; };
    uint32_t x0 = 0, x1 = 0;                        // column lane of L1^-1, of L2^-1
#pragma unroll 8
    for (int p = 0; p < 32; ++p) {
        const uint32_t l1 = (uint32_t)row(p);
        const uint32_t l2 = (uint32_t)(row(32 + p) >> 32);
        x0 |= (uint32_t)((((p == lane) ? 1 : 0) ^ __popc(l1 & x0)) & 1) << p;
        x1 |= (uint32_t)((((p == lane) ? 1 : 0) ^ __popc(l2 & x1)) & 1) << p;
    }
    // Y = C (column lane of L1^-1), C = rows 32..63, columns 0..31
    uint32_t y = 0;
#pragma unroll 8
    for (int p = 0; p < 32; ++p) y |= (uint32_t)(__popc((uint32_t)row(32 + p) & x0) & 1) << p;
    // rows of L2^-1 by ballot, then the lower-left column L2^-1 Y
    uint32_t z = 0;
    uint32_t r1lo = 0, r2lo = 0, r2hi = 0;
#pragma unroll 8
    for (int p = 0; p < 32; ++p) {
        const uint32_t l2inv_p = __ballot_sync(FULL, (x1 >> p) & 1u);
        z |= (uint32_t)(__popc(l2inv_p & y) & 1) << p;
    }
    // row p of L^-1: [L1^-1 row p | 0]; row 32 + p: [lower-left row p | L2^-1 row p]
#pragma unroll 8
    for (int p = 0; p < 32; ++p) {
        const uint32_t a = __ballot_sync(FULL, (x0 >> p) & 1u);
        const uint32_t b = __ballot_sync(FULL, (z >> p) & 1u);
        const uint32_t c = __ballot_sync(FULL, (x1 >> p) & 1u);
        if (lane == p) { r1lo = a; r2lo = b; r2hi = c; }
    }
    const uint64_t v0 = (uint64_t)r1lo, v1 = ((uint64_t)r2hi << 32) | r2lo;
    if (lane < n) {
        out[lane] = v0;
        if (out2) out2[lane] = v0;
    }
    if (lane + 32 < n) {
        out[lane + 32] = v1;
        if (out2) out2[lane + 32] = v1;
    }
}

// U11^-1 by one warp from the pivot rows of a finished search: U11[p][q] is
// bit qbar[q] of E[p] (unit upper triangular); reversing the order of rows
// and columns makes it unit lower triangular, inverted in 32 x 32 blocks.
// sU, sUi: 64-word scratch.  Writes row p of U11^-1 to out[p] for p < rbar.
__device__ __forceinline__ void warp_upper_inverse(const PanelShared &sh, int rbar, uint64_t *sU, uint64_t *sUi,
                                                   uint64_t *out)
{
    const int lane = threadIdx.x & 31;
    for (int p = lane; p < KS; p += 32) {
        uint64_t u = 0;
        if (p < rbar) {
            const uint64_t e = sh.E[p];
#pragma unroll 16
            for (int q = 0; q < KS; ++q) u |= (q < rbar ? ((e >> (sh.j[q] & 63)) & 1ull) : 0ull) << q;
        } else {
            u = 1ull << p;
        }
        sU[63 - p] = __brevll(u);                       // row 63 - p of the reversed matrix
    }
    __syncwarp();
    warp_lower_inverse_blocked(sU, KS, sUi);
    __syncwarp();
    for (int p = lane; p < rbar; p += 32) out[p] = __brevll(sUi[63 - p]);
}

}  // namespace gf2
