// kernels_panel.cu -- pivot search of one 64-column stripe and the per-row
// preparation of the stripe's trailing update.
//
// Block-iterative PLE (Section 3.2, Algorithm 2), one stripe of KS = 64
// columns starting at column c, rows from the current rank r:
//
//   panel_kernel  PartialPle of the stripe (Algorithm 1): column-wise search
//                 for pivots (leftmost column, first row in the current
//                 order), rows exchanged by swaps recorded LAPACK-style in P.
//                 Rows are not moved in memory here; the kernel only decides
//                 the pivots, the swap sequence and where each affected row's
//                 content currently lives.
//   prep_kernel   For every row at a position >= r: its coefficient vector v
//                 with respect to the stripe's echelon pivot rows E11 (the L
//                 bits, written in place at columns r .. r+rbar-1, Algorithm
//                 2's "compress L"), and the table index w = v * L11^-1 that
//                 selects the combination of the raw pivot rows to add
//                 (Section 3.2: A22 += L21 * A12 after A12 <- L11^-1 A12, here
//                 folded into the index).  Rows touched by the swaps are
//                 staged in S so that the update reads no row another CTA
//                 writes.
//
// Laziness (Algorithm 1) on a GPU: the pivot search only reads the stripe
// word of rows it inspects.  The fast path holds a window of up to 128 rows
// in the registers of one warp, bit-sliced: lane l owns columns l and l+32 as
// 128-row masks.  A pivot step is then one shuffle of column j, one find-
// first-set for the pivot row, and a handful of mask operations per lane for
// the row exchange and the elimination below the pivot; the L coefficients
// are kept the same way (one 128-row mask per pivot), and E11 / L11 come out
// by ballot at the end.  The window is exact whenever every pivot column
// finds its row inside it (or it holds all remaining rows).  Otherwise the
// block-wide path redoes the stripe over all remaining rows.
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

__global__ void init_ple_kernel(int64_t *P, int64_t *Q, int64_t m, int64_t qn, int32_t *map,
                                int64_t *r_dev)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (i == 0) *r_dev = 0;
    for (; i < m; i += stride) {
        P[i] = i;
        if (map) map[i] = -1;
        if (i < qn) Q[i] = -1;
    }
}

cudaError_t launch_init_ple(cudaStream_t st, int64_t *P, int64_t *Q, int64_t m, int64_t qn,
                            int32_t *map, int64_t *r_dev, int num_sms)
{
    int64_t blocks = (m + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 8 * num_sms) blocks = 8 * num_sms;
    init_ple_kernel<<<(int)blocks, 256, 0, st>>>(P, Q, m, qn, map, r_dev);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(PANEL_THREADS)
panel_kernel(const uint64_t *__restrict__ A, int64_t m, int64_t ld, int64_t npiv, int s,
             StripeDesc *descs, int64_t *r_dev, int64_t *P, int64_t *Q, int32_t *map,
             PanelScratch gs, int32_t *fallbacks)
{
    __shared__ uint64_t sh_E[KS], sh_L[KS];
    __shared__ int32_t sh_t[KS];
    __shared__ uint8_t sh_j[KS];
    __shared__ int32_t sh_Soff[SMAX];
    __shared__ int64_t sh_Ssrc[SMAX];
    __shared__ int32_t sh_perm[PANEL_WIN];
    __shared__ int sh_fail, sh_rbar, sh_nS, sh_maxpos, sh_best;
    __shared__ unsigned long long sh_colmask;

    StripeDesc *d = descs + s;
    const int64_t r = *r_dev;
    const int c = s * KS;
    const int64_t rows = m - r;
    const int keff = (int)min((int64_t)KS, npiv - (int64_t)c);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t cw = c >> 6;

    if (rows <= 0 || keff <= 0) {
        if (tid == 0) {
            d->r = r; d->rbar = 0; d->c = c; d->nS = 0; d->maxpos = -1; d->tier = 0;
        }
        return;
    }
    // ---------------- fast path: one warp, bit-sliced window of up to 128 rows
    if (warp == 0) {
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
        for (int x = lane; x < PANEL_WIN; x += 32) sh_perm[x] = x;
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
                sh_t[p] = t;
                sh_j[p] = (uint8_t)j;
                const int a = sh_perm[p];
                sh_perm[p] = sh_perm[t];
                sh_perm[t] = a;
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
                    sh_E[q0] = ((uint64_t)e01 << 32) | e00;
                    sh_L[q0] = ((((uint64_t)f01 << 32) | f00)) & ((q0 == 0) ? 0ull : (~0ull >> (64 - q0)));
                }
                if (q1 < p) {
                    sh_E[q1] = ((uint64_t)e11 << 32) | e10;
                    sh_L[q1] = ((((uint64_t)f11 << 32) | f10)) & (~0ull >> (64 - q1));
                }
            }
            __syncwarp();
            // staged rows: pivot rows first, then rows displaced into [p, tmax]
            for (int k = lane; k < p; k += 32) { sh_Soff[k] = k; sh_Ssrc[k] = r + sh_perm[k]; }
            int base = p;
            for (int b0 = p; b0 <= tmax; b0 += 32) {
                const int sl = b0 + lane;
                const bool mv = sl <= tmax && sh_perm[sl] != sl;
                const unsigned bm = __ballot_sync(0xffffffffu, mv);
                if (mv) {
                    const int k = base + __popc(bm & ((1u << lane) - 1u));
                    sh_Soff[k] = sl;
                    sh_Ssrc[k] = r + sh_perm[sl];
                }
                base += __popc(bm);
            }
            if (lane == 0) { sh_nS = base; sh_maxpos = max(p - 1, tmax); }
        }
        if (lane == 0) { sh_fail = fail ? 1 : 0; sh_rbar = p; }
    }
    __syncthreads();

    // ---------------- block-wide path over all remaining rows
    if (sh_fail) {
        const int nthr = blockDim.x;
        if (tid == 0) { sh_colmask = 0; if (fallbacks) atomicAdd(fallbacks, 1); }
        __syncthreads();
        unsigned long long orv = 0;
        for (int64_t sl = tid; sl < rows; sl += nthr) {
            const uint64_t v = A[(r + sl) * ld + cw];
            gs.val[sl] = v;
            gs.lb[sl] = 0;
            gs.src[sl] = (int32_t)sl;
            orv |= v;
        }
        const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)orv);
        const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(orv >> 32));
        if (lane == 0) atomicOr(&sh_colmask, ((unsigned long long)hi << 32) | lo);
        __syncthreads();
        // a column that is zero in every remaining row stays zero in every
        // combination of them, so it can never hold a pivot
        const uint64_t colmask = sh_colmask;
        int p = 0, tmax = -1;
        for (int j = 0; j < keff && p < rows; ++j) {
            if (!((colmask >> j) & 1ull)) continue;
            __syncthreads();
            if (tid == 0) sh_best = INT_MAX;
            __syncthreads();
            for (int64_t base = p; base < rows; base += nthr) {
                const int64_t sl = base + tid;
                const bool hit = sl < rows && ((gs.val[sl] >> j) & 1ull);
                if (__syncthreads_or(hit)) {
                    if (hit) atomicMin(&sh_best, (int)sl);
                    __syncthreads();
                    break;
                }
            }
            const int t = sh_best;
            if (t == INT_MAX) continue;
            __syncthreads();
            if (tid == 0) {
                const uint64_t tv = gs.val[t], tl = gs.lb[t];
                const int32_t ts = gs.src[t];
                gs.val[t] = gs.val[p]; gs.lb[t] = gs.lb[p]; gs.src[t] = gs.src[p];
                gs.val[p] = tv; gs.lb[p] = tl; gs.src[p] = ts;
                sh_t[p] = t; sh_j[p] = (uint8_t)j; sh_E[p] = tv; sh_L[p] = tl;
            }
            __syncthreads();
            const uint64_t pv = sh_E[p];
            const uint64_t bitp = 1ull << p;
            for (int64_t sl = p + 1 + tid; sl < rows; sl += nthr) {
                const uint64_t v = gs.val[sl];
                if ((v >> j) & 1ull) { gs.val[sl] = v ^ pv; gs.lb[sl] |= bitp; }
            }
            tmax = max(tmax, t);
            ++p;
        }
        __syncthreads();
        if (tid == 0) { sh_rbar = p; sh_nS = p; sh_maxpos = max(p - 1, tmax); }
        for (int k = tid; k < p; k += nthr) { sh_Soff[k] = k; sh_Ssrc[k] = r + gs.src[k]; }
        __syncthreads();
        for (int64_t sl = p + tid; sl <= tmax; sl += nthr) {
            if (gs.src[sl] != (int32_t)sl) {
                const int k = atomicAdd(&sh_nS, 1);
                sh_Soff[k] = (int32_t)sl;
                sh_Ssrc[k] = r + gs.src[sl];
            }
        }
        __syncthreads();
    }

    // ---------------- outputs
    const int rbar = sh_rbar;
    if (warp == 1) {
        // U11^-1 for the RREF recovery, U11[p][q] = E11[p] at column qbar[q]
        // (unit upper triangular): lane-parallel backward substitution per
        // column, rows collected by ballot.  Runs beside warp 0's L11^-1.
        __shared__ uint64_t sU[KS];
        for (int p = lane; p < rbar; p += 32) {
            const uint64_t e = sh_E[p];
            uint64_t u = 0;
            for (int q = 0; q < rbar; ++q) u |= ((e >> sh_j[q]) & 1ull) << q;
            sU[p] = u;
        }
        __syncwarp();
        uint64_t x0 = 0, x1 = 0;
        for (int p = rbar - 1; p >= 0; --p) {
            const uint64_t up = sU[p];
            x0 |= (uint64_t)((((p == lane) ? 1 : 0) ^ __popcll(up & x0)) & 1) << p;
            x1 |= (uint64_t)((((p == lane + 32) ? 1 : 0) ^ __popcll(up & x1)) & 1) << p;
        }
        for (int p = 0; p < rbar; ++p) {
            const unsigned lo = __ballot_sync(0xffffffffu, (x0 >> p) & 1ull);
            const unsigned hi = __ballot_sync(0xffffffffu, (x1 >> p) & 1ull);
            if (lane == 0) d->Minv[p] = ((uint64_t)hi << 32) | lo;
        }
    }
    if (warp == 0) {
        // L11^-1 column by column (lane owns columns lane and lane + 32):
        // forward substitution L x = e_col, then rows by ballot.
        uint64_t x0 = 0, x1 = 0;
        for (int p = 0; p < rbar; ++p) {
            const uint64_t Lp = sh_L[p];
            x0 |= (uint64_t)((((p == lane) ? 1 : 0) ^ __popcll(Lp & x0)) & 1) << p;
            x1 |= (uint64_t)((((p == lane + 32) ? 1 : 0) ^ __popcll(Lp & x1)) & 1) << p;
        }
        for (int p = 0; p < rbar; ++p) {
            const unsigned lo = __ballot_sync(0xffffffffu, (x0 >> p) & 1ull);
            const unsigned hi = __ballot_sync(0xffffffffu, (x1 >> p) & 1ull);
            if (lane == 0) d->Linv[p] = ((uint64_t)hi << 32) | lo;
        }
    }
    for (int p = tid; p < rbar; p += blockDim.x) {
        P[r + p] = r + sh_t[p];
        Q[r + p] = c + sh_j[p];
        d->E11[p] = sh_E[p];
        d->L11[p] = sh_L[p];
        d->qbar[p] = sh_j[p];
    }
    const int nS = sh_nS;
    for (int k = tid; k < nS; k += blockDim.x) {
        d->S_off[k] = sh_Soff[k];
        d->S_src[k] = sh_Ssrc[k];
        map[r + sh_Soff[k]] = s * 256 + k;
    }
    if (tid == 0) {
        d->r = r; d->rbar = rbar; d->c = c; d->nS = nS; d->maxpos = sh_maxpos;
        d->tier = sh_fail ? 2 : 1;
        *r_dev = r + rbar;
    }
}

cudaError_t launch_panel(cudaStream_t st, uint64_t *A, int64_t m, int64_t ld, int64_t npiv, int s,
                         StripeDesc *descs, int64_t *r_dev, int64_t *P, int64_t *Q, int32_t *map,
                         PanelScratch gs, int32_t *fallbacks)
{
    panel_kernel<<<1, PANEL_THREADS, 0, st>>>(A, m, ld, npiv, s, descs, r_dev, P, Q, map, gs,
                                              fallbacks);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// prep

// Write the L bits v at columns [r, r + nv) and the stripe word es at word cw
// of one row; the old L bits below column r are kept.  Words strictly between
// the L bits and the stripe are zero already and stay zero.
__device__ __forceinline__ void write_lregion(uint64_t *row, int64_t r, int64_t cw, int rbar,
                                              uint64_t v, uint64_t es)
{
    const int64_t wr = r >> 6;
    const int64_t wl = (r + rbar - 1) >> 6;
    for (int64_t w = wr; w <= wl; ++w) {
        const int64_t off = r - (w << 6);
        uint64_t part = (off >= 0) ? (v << off) : (v >> (-off));
        const uint64_t keep = (w == wr) ? (row[w] & ((1ull << (r & 63)) - 1ull)) : 0ull;
        if (w == cw) part |= es;
        row[w] = keep | part;
    }
    if (cw > wl) row[cw] = es;
}

constexpr int PREP_THREADS = 256;
constexpr int PREP_STAGE_BLOCKS = SMAX;   // one block per staged row
constexpr int PREP_FIRST_ROW_BLOCK = PREP_STAGE_BLOCKS;

__global__ void __launch_bounds__(PREP_THREADS)
prep_kernel(uint64_t *A, int64_t m, int64_t ld, int64_t W, int s, StripeDesc *descs,
            const int32_t *map, uint64_t *S, int64_t ldS, uint64_t *IDX, int32_t *err)
{
    StripeDesc *d = descs + s;
    const int rbar = d->rbar;
    if (rbar == 0) return;
    const int64_t r = d->r;
    const int64_t cw = d->c >> 6;
    const int nS = d->nS;
    const int maxpos = d->maxpos;
    __shared__ uint64_t sE[KS], sLinv[KS];
    __shared__ int sq[KS];
    for (int i = threadIdx.x; i < rbar; i += blockDim.x) {
        sE[i] = d->E11[i];
        sLinv[i] = d->Linv[i];
        sq[i] = d->qbar[i];
    }
    __syncthreads();

    if (blockIdx.x < PREP_STAGE_BLOCKS) {
        // staged rows: copy the whole source row, then fix its L region
        for (int k = blockIdx.x; k < nS; k += PREP_STAGE_BLOCKS) {   // at most one per block
            const uint64_t *src = A + d->S_src[k] * ld;
            uint64_t *dst = S + (int64_t)k * ldS;
            for (int64_t w = threadIdx.x; w < W; w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            if (threadIdx.x == 0) {
                const int64_t pos = r + d->S_off[k];
                uint64_t v, es, ix;
                if (k < rbar) {
                    v = d->L11[k];
                    es = sE[k];
                    ix = sLinv[k] ^ (1ull << k);
                } else {
                    uint64_t sw = dst[cw];
                    v = 0;
                    for (int p = 0; p < rbar; ++p) {
                        const uint64_t bit = (sw >> sq[p]) & 1ull;
                        sw ^= sE[p] & (0ull - bit);
                        v |= bit << p;
                    }
                    if (sw && err) atomicExch(err, 1);
                    es = 0;
                    ix = 0;
                    for (int p = 0; p < rbar; ++p) ix ^= sLinv[p] & (0ull - ((v >> p) & 1ull));
                }
                write_lregion(dst, r, cw, rbar, v, es);
                IDX[pos] = ix;
            }
            __syncthreads();
        }
        return;
    }
    const int64_t stride = (int64_t)(gridDim.x - PREP_FIRST_ROW_BLOCK) * blockDim.x;
    for (int64_t i = r + (int64_t)(blockIdx.x - PREP_FIRST_ROW_BLOCK) * blockDim.x + threadIdx.x;
         i < m; i += stride) {
        if (i - r <= maxpos) {
            const int mv = map[i];
            if (mv >= 0 && (mv >> 8) == s) continue;       // staged row
        }
        uint64_t *row = A + i * ld;
        uint64_t sw = row[cw];
        uint64_t v = 0;
        for (int p = 0; p < rbar; ++p) {
            const uint64_t bit = (sw >> sq[p]) & 1ull;
            sw ^= sE[p] & (0ull - bit);
            v |= bit << p;
        }
        if (sw && err) atomicExch(err, 1);
        uint64_t ix = 0;
        for (int p = 0; p < rbar; ++p) ix ^= sLinv[p] & (0ull - ((v >> p) & 1ull));
        write_lregion(row, r, cw, rbar, v, 0ull);
        IDX[i] = ix;
    }
}

cudaError_t launch_prep(cudaStream_t st, uint64_t *A, int64_t m, int64_t ld, int64_t W, int s,
                        StripeDesc *descs, const int32_t *map, uint64_t *S, int64_t ldS,
                        uint64_t *IDX, int32_t *err, int num_sms)
{
    int64_t blocks = (m + PREP_THREADS - 1) / PREP_THREADS;
    if (blocks < 1) blocks = 1;
    if (blocks > 4 * num_sms) blocks = 4 * num_sms;
    prep_kernel<<<(int)(blocks + PREP_FIRST_ROW_BLOCK), PREP_THREADS, 0, st>>>(
        A, m, ld, W, s, descs, map, S, ldS, IDX, err);
    return cudaGetLastError();
}

}  // namespace gf2
