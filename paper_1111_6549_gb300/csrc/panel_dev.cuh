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
    // transposed window path (panel_window_t): rows of L11^-1 and U11^-1
    uint64_t Linv[KS], Minv[KS];
};

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
                                             int64_t cw, int64_t rows, int keff, PanelShared &sh)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int Wn = (int)min(rows, (int64_t)PANEL_WIN);
    uint64_t R[4], Lc[4];
    int org[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int sl = b * 32 + lane;
        R[b] = (sl < Wn) ? A[(r + sl) * ld + cw] : 0ull;
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
// lane + 32), rows collected by ballot; lane 0 writes out[p] (and out2[p]).
__device__ __forceinline__ void warp_lower_inverse(const uint64_t *Lrows, int rbar, uint64_t *out,
                                                   uint64_t *out2 = nullptr)
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
        if (lane == 0) {
            const uint64_t v = ((uint64_t)hi << 32) | lo;
            out[p] = v;
            if (out2) out2[p] = v;
        }
    }
}

// Column `lane` of a 32 x 32 bit block: lane i passes row i (bit j = entry
// (i, j)), lane l gets bit i = entry (i, l).  Five butterfly exchanges of
// halving sub-blocks.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x)
{
    const int lane = threadIdx.x & 31;
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int d = 16 >> k;
        const uint32_t m = masks[k];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, d);
        x = (lane & d) ? (((y >> d) & m) | (x & ~m)) : ((x & m) | ((y & m) << d));
    }
    return x;
}

// 64 x 64 bit matrix held by columns (lane l: columns l and l + 32, bit p =
// row p) -> by rows (lane l: rows l and l + 32, bit q = column q).
__device__ __forceinline__ void warp_transpose64(uint64_t c0, uint64_t c1, uint64_t &r0, uint64_t &r1)
{
    const uint32_t a = warp_transpose32((uint32_t)c0), b = warp_transpose32((uint32_t)c1);
    const uint32_t c = warp_transpose32((uint32_t)(c0 >> 32)), e = warp_transpose32((uint32_t)(c1 >> 32));
    r0 = ((uint64_t)b << 32) | a;
    r1 = ((uint64_t)e << 32) | c;
}

// A set of the 128 window slots: lo = slots 0..63, hi = slots 64..127.
struct SlotMask {
    uint64_t lo, hi;
};

// Exchange slots p (< 64) and t (> p) in m; pt = the mask of both slots.
__device__ __forceinline__ void slot_swap(SlotMask &m, int p, int t, const SlotMask &pt)
{
    const uint64_t bp = (m.lo >> p) & 1ull;
    const uint64_t bt = t < 64 ? ((m.lo >> t) & 1ull) : ((m.hi >> (t - 64)) & 1ull);
    const uint64_t sel = 0ull - (bp ^ bt);
    m.lo ^= pt.lo & sel;
    m.hi ^= pt.hi & sel;
}

// Transposed fast path, called by one whole warp: the same search as
// panel_window (Algorithm 1 on a window of up to 128 rows), with the window
// held by columns -- lane l owns the slot masks of columns l and l + 32 --
// so that a pivot step is one broadcast of column j's mask, a find-first-set
// and a few mask operations per lane.  Besides E, L, t, j and the staged-row
// list it leaves L11^-1 and U11^-1 in sh.Linv / sh.Minv, taken from masks
// kept during the elimination:
//   * L11: pivot q's mask of the slots it eliminated (the rows below it);
//   * L11^-1: per slot, which earlier pivot rows' raw contents its content
//     holds beside its own (V); at its selection, pivot p's row is its own raw
//     row plus V_p, so row p of L11^-1 is e_p + V_p;
//   * U11^-1: each pivot also clears its column from the earlier pivot rows
//     (their contents become the fully reduced rows, GaussSubmatrix); the set
//     it cleared is column q of U11^-1 above the diagonal.
// The pivot rows' echelon form E (before that reduction) is taken by ballot
// at each selection.  Sets sh.fail exactly when panel_window would.
__device__ __forceinline__ void panel_window_t(const uint64_t *__restrict__ A, int64_t r, int64_t ld,
                                               int64_t cw, int64_t rows, int keff, PanelShared &sh)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const int Wn = (int)min(rows, (int64_t)PANEL_WIN);
    uint64_t R[4];
    int org[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int sl = b * 32 + lane;
        R[b] = (sl < Wn) ? A[(r + sl) * ld + cw] : 0ull;
        org[b] = sl;
    }
    // columns: Mc[h] = slots holding column 32 h + lane
    SlotMask Mc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint64_t s0 = warp_transpose32((uint32_t)(R[0] >> (32 * h)));
        const uint64_t s1 = warp_transpose32((uint32_t)(R[1] >> (32 * h)));
        const uint64_t s2 = warp_transpose32((uint32_t)(R[2] >> (32 * h)));
        const uint64_t s3 = warp_transpose32((uint32_t)(R[3] >> (32 * h)));
        Mc[h].lo = s0 | (s1 << 32);
        Mc[h].hi = s2 | (s3 << 32);
    }
    SlotMask LM[2] = {{0, 0}, {0, 0}}, VM[2] = {{0, 0}, {0, 0}};   // pivots lane, lane + 32
    uint64_t UM[2] = {0, 0}, Er[2] = {0, 0};
    int p = 0, tmax = -1;
    bool fail = false;
    for (int j = 0; j < keff && p < Wn; ++j) {
        const int jh = j >> 5, jl = j & 31;
        const SlotMask src = jh ? Mc[1] : Mc[0];
        SlotMask Mj;
        Mj.lo = __shfl_sync(FULL, src.lo, jl);
        Mj.hi = __shfl_sync(FULL, src.hi, jl);
        const uint64_t clo = Mj.lo & (~0ull << p);        // p < 64: slots >= p
        if (!(clo | Mj.hi)) {
            if (Wn < rows) { fail = true; break; }       // the pivot may lie outside the window
            continue;                                    // column j has no pivot
        }
        const int t = clo ? __ffsll((long long)clo) - 1 : 64 + __ffsll((long long)Mj.hi) - 1;
        if (t != p) {
            SlotMask pt;
            pt.lo = (1ull << p) | (t < 64 ? (1ull << t) : 0ull);
            pt.hi = t < 64 ? 0ull : (1ull << (t - 64));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                slot_swap(Mc[h], p, t, pt);
                slot_swap(LM[h], p, t, pt);
                slot_swap(VM[h], p, t, pt);
            }
            slot_swap(Mj, p, t, pt);
            const int op = __shfl_sync(FULL, pick4(org, p >> 5), p & 31);
            const int ot = __shfl_sync(FULL, pick4(org, t >> 5), t & 31);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (32 * b + lane == p) org[b] = ot;
                if (32 * b + lane == t) org[b] = op;
            }
        }
        // the pivot row (now slot p): its echelon word, by ballot
        const unsigned elo = __ballot_sync(FULL, (unsigned)(Mc[0].lo >> p) & 1u);
        const unsigned ehi = __ballot_sync(FULL, (unsigned)(Mc[1].lo >> p) & 1u);
        SlotMask below;
        below.lo = Mj.lo & ((p == 63) ? 0ull : (~0ull << (p + 1)));
        below.hi = Mj.hi;
        const uint64_t above = Mj.lo & ((1ull << p) - 1ull);
        // clear column j from every other slot holding it: the columns the
        // pivot row holds take (below + above); V of the rows below takes
        // V_p + e_p
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint64_t sc = 0ull - ((Mc[h].lo >> p) & 1ull);
            Mc[h].lo ^= (below.lo | above) & sc;
            Mc[h].hi ^= below.hi & sc;
            const uint64_t sv = 0ull - ((VM[h].lo >> p) & 1ull);
            VM[h].lo ^= below.lo & sv;
            VM[h].hi ^= below.hi & sv;
        }
        if (lane == (p & 31)) {
            const int h = p >> 5;
            const uint64_t e = ((uint64_t)ehi << 32) | elo;
            if (h == 0) { VM[0].lo ^= below.lo; VM[0].hi ^= below.hi; LM[0] = below; UM[0] = above; Er[0] = e; }
            else        { VM[1].lo ^= below.lo; VM[1].hi ^= below.hi; LM[1] = below; UM[1] = above; Er[1] = e; }
        }
        if (lane == 0) {
            sh.t[p] = t;
            sh.j[p] = (uint8_t)j;
        }
        tmax = max(tmax, t);
        ++p;
    }
    if (!fail) {
        // rows of L11 (bit q < p: pivot q cleared row p), of L11^-1 (e_p + V_p)
        // and of U11^-1 (e_p + the later pivots that cleared their column
        // from row p), by transposing the per-pivot masks
        uint64_t l0, l1, v0, v1, u0, u1;
        warp_transpose64(LM[0].lo, LM[1].lo, l0, l1);
        warp_transpose64(VM[0].lo, VM[1].lo, v0, v1);
        warp_transpose64(UM[0] | (1ull << lane), UM[1] | (1ull << (lane + 32)), u0, u1);
        const uint64_t below_diag0 = (lane == 0) ? 0ull : (~0ull >> (64 - lane));
        const uint64_t below_diag1 = ~0ull >> (32 - lane);
        if (lane < p) {
            sh.E[lane] = Er[0];
            sh.L[lane] = l0 & below_diag0;
            sh.Linv[lane] = ((v0 & below_diag0) | (1ull << lane));
            sh.Minv[lane] = u0 & ~below_diag0 & ((p == 64) ? ~0ull : ((1ull << p) - 1ull));
        }
        if (lane + 32 < p) {
            sh.E[lane + 32] = Er[1];
            sh.L[lane + 32] = l1 & below_diag1;
            sh.Linv[lane + 32] = ((v1 & below_diag1) | (1ull << (lane + 32)));
            sh.Minv[lane + 32] = u1 & ~below_diag1 & ((p == 64) ? ~0ull : ((1ull << p) - 1ull));
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

}  // namespace gf2
