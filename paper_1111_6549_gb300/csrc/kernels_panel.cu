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
// word of rows it inspects.  The fast path holds a window of 32*PANEL_G rows
// in the registers of one warp and uses ballot / ffs / shuffles; it is exact
// whenever every pivot column finds its row inside the window (or the window
// holds all remaining rows).  Otherwise the block-wide path redoes the stripe
// over all remaining rows.
#include "common.cuh"

#include <climits>

namespace gf2 {

template <int G>
__device__ __forceinline__ uint64_t sel(const uint64_t (&a)[G], int g)
{
    uint64_t v = a[0];
#pragma unroll
    for (int i = 1; i < G; ++i) v = (g == i) ? a[i] : v;
    return v;
}
template <int G>
__device__ __forceinline__ int sel(const int (&a)[G], int g)
{
    int v = a[0];
#pragma unroll
    for (int i = 1; i < G; ++i) v = (g == i) ? a[i] : v;
    return v;
}
template <int G, typename T>
__device__ __forceinline__ void put(T (&a)[G], int g, T v)
{
#pragma unroll
    for (int i = 0; i < G; ++i)
        if (g == i) a[i] = v;
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
    const int Wn = (int)min(rows, (int64_t)(32 * PANEL_G));

    // ---------------- fast path: one warp, window of Wn rows in registers
    if (warp == 0) {
        uint64_t val[PANEL_G], lb[PANEL_G];
        int so[PANEL_G];
#pragma unroll
        for (int g = 0; g < PANEL_G; ++g) {
            const int sl = g * 32 + lane;
            val[g] = (sl < Wn) ? A[(r + sl) * ld + cw] : 0ull;
            lb[g] = 0;
            so[g] = sl;
        }
        int p = 0, tmax = -1;
        bool fail = false;
        for (int j = 0; j < keff && p < Wn; ++j) {
            int t = -1;
#pragma unroll
            for (int g = 0; g < PANEL_G; ++g) {
                const int sl = g * 32 + lane;
                const bool cand = (sl >= p) && (sl < Wn) && ((val[g] >> j) & 1ull);
                const unsigned b = __ballot_sync(0xffffffffu, cand);
                if (t < 0 && b) t = g * 32 + __ffs(b) - 1;
            }
            if (t < 0) {
                if (Wn < rows) { fail = true; break; }   // the pivot may lie outside the window
                continue;                                // column j has no pivot
            }
            const int gt = t >> 5, lt = t & 31, gp = p >> 5, lp = p & 31;
            const uint64_t pv = __shfl_sync(0xffffffffu, sel(val, gt), lt);
            const uint64_t pl = __shfl_sync(0xffffffffu, sel(lb, gt), lt);
            const int ps = __shfl_sync(0xffffffffu, sel(so, gt), lt);
            const uint64_t xv = __shfl_sync(0xffffffffu, sel(val, gp), lp);
            const uint64_t xl = __shfl_sync(0xffffffffu, sel(lb, gp), lp);
            const int xs = __shfl_sync(0xffffffffu, sel(so, gp), lp);
            // swap positions p and t: the pivot row moves to p, the row at p to t
            if (lane == lt) { put(val, gt, xv); put(lb, gt, xl); put(so, gt, xs); }
            if (lane == lp) { put(val, gp, pv); put(lb, gp, pl); put(so, gp, ps); }
            if (lane == 0) { sh_t[p] = t; sh_j[p] = (uint8_t)j; sh_E[p] = pv; sh_L[p] = pl; }
            tmax = max(tmax, t);
            const uint64_t bitp = 1ull << p;
#pragma unroll
            for (int g = 0; g < PANEL_G; ++g) {
                const int sl = g * 32 + lane;
                if (sl > p && sl < Wn && ((val[g] >> j) & 1ull)) { val[g] ^= pv; lb[g] |= bitp; }
            }
            ++p;
        }
        if (!fail) {
            // staged rows: pivot rows first (slot k = position offset k), then
            // displaced rows (slots in [p, tmax] whose content came from elsewhere)
#pragma unroll
            for (int g = 0; g < PANEL_G; ++g) {
                const int sl = g * 32 + lane;
                if (sl < p) { sh_Soff[sl] = sl; sh_Ssrc[sl] = r + so[g]; }
            }
            int base = p;
#pragma unroll
            for (int g = 0; g < PANEL_G; ++g) {
                const int sl = g * 32 + lane;
                const bool mv = sl >= p && sl <= tmax && so[g] != sl;
                const unsigned b = __ballot_sync(0xffffffffu, mv);
                if (mv) {
                    const int k = base + __popc(b & ((1u << lane) - 1u));
                    sh_Soff[k] = sl;
                    sh_Ssrc[k] = r + so[g];
                }
                base += __popc(b);
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
constexpr int PREP_STAGE_BLOCKS = 32;

__global__ void __launch_bounds__(PREP_THREADS)
prep_kernel(uint64_t *A, int64_t m, int64_t ld, int64_t W, int s, const StripeDesc *descs,
            const int32_t *map, uint64_t *S, int64_t ldS, uint64_t *IDX, int32_t *err)
{
    const StripeDesc *d = descs + s;
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
        for (int k = blockIdx.x; k < nS; k += PREP_STAGE_BLOCKS) {
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
    const int64_t stride = (int64_t)(gridDim.x - PREP_STAGE_BLOCKS) * blockDim.x;
    for (int64_t i = r + (int64_t)(blockIdx.x - PREP_STAGE_BLOCKS) * blockDim.x + threadIdx.x;
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
                        const StripeDesc *descs, const int32_t *map, uint64_t *S, int64_t ldS,
                        uint64_t *IDX, int32_t *err, int num_sms)
{
    int64_t blocks = (m + PREP_THREADS - 1) / PREP_THREADS;
    if (blocks < 1) blocks = 1;
    if (blocks > 4 * num_sms) blocks = 4 * num_sms;
    prep_kernel<<<(int)(blocks + PREP_STAGE_BLOCKS), PREP_THREADS, 0, st>>>(
        A, m, ld, W, s, descs, map, S, ldS, IDX, err);
    return cudaGetLastError();
}

}  // namespace gf2
