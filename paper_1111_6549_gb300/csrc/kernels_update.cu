// kernels_update.cu -- the tabulated trailing update (the hot loop).
//
// For every row i of a row range and every word of a column range:
//     row_i ^= T_0[idx_i byte 0] ^ T_1[idx_i byte 1] ^ ... ^ T_7[idx_i byte 7]
// where T_t holds all 256 combinations of the eight generator rows
// 8t .. 8t+7 (Section 3.2: "a table T of all 2^k linear combinations ...
// for each row of A22 we perform one row addition from the table"; Appendix
// A, Algorithms 5 and 6; eight tables of k = 8 bits clear 64 columns per
// pass, as the implementation's multiple Gray-code tables of Section 4 do).
// The same kernel serves three callers:
//   UPD_PLE   rows at positions >= r of Algorithm 2, right of the stripe; the
//             generators are the stripe's raw pivot rows (staged in S) and
//             the index is w = v L11^-1, so one lookup applies both
//             A12 <- L11^-1 A12 (pivot rows) and A22 += L21 A12 (the rest).
//   UPD_RREF  rows above a pivot block during RREF recovery; generators are
//             the block's reduced rows indexed by pivot column, the index is
//             the row's raw stripe word.
//   UPD_MUL   C ^= A[:, 64 kc .. 64 kc + 63] B[64 kc .. 64 kc + 63, :].
//
// GB300 mapping.  The kernel is bound by HBM: each 64-bit word of the
// trailing block is read and written once per stripe.  A persistent grid of
// one CTA per SM splits the (column tile x row) space evenly; each CTA builds
// the eight tables for its column tile of TW = 8 words (64 bytes per row) in
// 128 KiB of shared memory and streams its rows through them.  Tables are
// built by doubling inside 32-entry Gray-code segments (255 additions per
// table and word, the count of Algorithm 6).  Two tables share one 128-byte
// line (table 2a in bytes 0..63, table 2a+1 in bytes 64..127); the two rows
// served by one 8-lane quarter-warp visit the tables in the orders
// t and t^1, so every 16-byte lookup phase hits 32 distinct banks whatever
// the indices are.
#include "tables_dev.cuh"

namespace gf2 {

template <bool VEC>
__global__ void __launch_bounds__(UPD_THREADS, 1) update_kernel(UpdArgs a)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint64_t T[];
    __shared__ const uint64_t *sGen[KS];

    int64_t row_lo, row_hi, w_lo;
    const int64_t W = a.W;
    int64_t r = 0;
    int maxpos = -1, nS = 0, rbar_m = 0;
    const StripeDesc *d = a.desc;
    if (a.mode == UPD_PLE) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        r = d->r;
        row_lo = r;
        row_hi = a.m;
        w_lo = (d->c >> 6) + (a.first_off > 0 ? a.first_off : 1);
        maxpos = d->maxpos;
        nS = d->nS;
        if (threadIdx.x < KS)
            sGen[threadIdx.x] = (threadIdx.x < rbar) ? a.S + threadIdx.x * a.ldS : nullptr;
    } else if (a.mode == UPD_RREF) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        row_lo = a.row_lo;                    // 0, or the first row of a block's own RREF
        row_hi = d->r;
        w_lo = max((int64_t)(d->c >> 6), a.w_lo);  // a.w_lo > 0: only a right part of the row
        if (threadIdx.x < KS) sGen[threadIdx.x] = nullptr;
        __syncthreads();
        if (threadIdx.x < rbar) sGen[d->qbar[threadIdx.x]] = a.A + (d->r + threadIdx.x) * a.ld;
    } else if (a.mode == UPD_M4RI) {
        rbar_m = d->rbar;
        if (rbar_m == 0) return;
        r = d->r;
        row_lo = 0;
        row_hi = a.m;
        w_lo = d->c >> 6;
        maxpos = d->maxpos;
        if (threadIdx.x < KS) sGen[threadIdx.x] = nullptr;
        __syncthreads();
        if (threadIdx.x < rbar_m) sGen[d->qbar[threadIdx.x]] = a.B + threadIdx.x * a.ldb;
    } else {
        row_lo = a.row_lo;
        row_hi = a.row_hi;
        w_lo = a.w_lo;
        if (threadIdx.x < KS)
            sGen[threadIdx.x] = (threadIdx.x < a.gen_count) ? a.B + threadIdx.x * a.ldb : nullptr;
    }
    __syncthreads();

    // M4RI: the pivot positions r .. r+rbar-1 take the reduced pivot rows
    if (a.mode == UPD_M4RI) {
        for (int p = blockIdx.x; p < rbar_m; p += gridDim.x)
            for (int64_t w = w_lo + threadIdx.x; w < W; w += blockDim.x) a.A[(r + p) * a.ld + w] = a.B[p * a.ldb + w];
    }
    // PLE: staged rows get their left part (old L bits, new L bits, stripe)
    // and the words past the updated range
    if (a.mode == UPD_PLE) {
        for (int k = blockIdx.x; k < nS; k += gridDim.x) {
            const uint64_t *src = a.S + (int64_t)k * a.ldS;
            uint64_t *dst = a.A + (r + d->S_off[k]) * a.ld;
            for (int64_t w = threadIdx.x; w < w_lo; w += blockDim.x) dst[w] = src[w];
            for (int64_t w = W + threadIdx.x; w < a.W_full; w += blockDim.x) dst[w] = src[w];
        }
    }

    const int64_t R = row_hi - row_lo;
    if (R <= 0 || w_lo >= W) return;
    const int64_t a0 = w_lo / TW, a1 = (W + TW - 1) / TW;
    const int64_t NT = a1 - a0;
    const int64_t U = NT * R;
    const int64_t u_beg = U * blockIdx.x / gridDim.x;
    const int64_t u_end = U * (blockIdx.x + 1) / gridDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.bytes)
        atomicAdd(a.bytes, (unsigned long long)(R * (W - w_lo) * 16));

    const int rs = threadIdx.x >> 2;        // row slot 0..127
    const int qd = threadIdx.x & 3;         // quad: words 2qd, 2qd+1 of the tile
    const int rho = rs & 1;                 // table visiting order t ^ rho
    constexpr int SLOTS = UPD_THREADS / 4;
    constexpr int RPT = UPD_ROWS_PER_THREAD;

    int64_t cur_tile = -1;
    for (int64_t u = u_beg; u < u_end;) {
        const int64_t tile = u / R;
        const int64_t rr0 = u - tile * R;
        const int64_t nrows = min(R - rr0, u_end - u);
        const int64_t wbase = (a0 + tile) * TW;
        if (tile != cur_tile) {
            __syncthreads();
            build_tables(T, sGen, wbase, W);
            __syncthreads();
            cur_tile = tile;
        }
        const int64_t w0 = wbase + 2 * qd;
        const bool lo_in = w0 >= w_lo && w0 < W;
        const bool hi_in = w0 + 1 >= w_lo && w0 + 1 < W;
        const uint64_t *Tq = T + 2 * qd;
        for (int64_t rb = 0; rb < nrows; rb += (int64_t)SLOTS * RPT) {
            int64_t ri[RPT];
            uint64_t ix[RPT], x0[RPT], x1[RPT];
            const uint64_t *src[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int64_t off = rb + (int64_t)k * SLOTS + rs;
                ri[k] = (off < nrows) ? row_lo + rr0 + off : -1;
                if (ri[k] >= r && ri[k] < r + rbar_m) ri[k] = -1;   // M4RI pivot positions
                src[k] = nullptr;
                ix[k] = 0;
                if (ri[k] >= 0) {
                    const int64_t i = ri[k];
                    ix[k] = a.idx[i * a.idx_stride];
                    const uint64_t *sp = a.A + i * a.ld;
                    if ((a.mode == UPD_PLE || a.mode == UPD_M4RI) && i >= r && i - r <= maxpos) {
                        const int mv = a.map[i];
                        if (mv >= 0 && (mv >> 8) == a.stripe) sp = a.S + (int64_t)(mv & 255) * a.ldS;
                    }
                    src[k] = sp;
                }
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                x0[k] = 0;
                x1[k] = 0;
                if (src[k]) {
                    if (VEC && lo_in && hi_in) {
                        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(src[k] + w0);
                        x0[k] = v.x;
                        x1[k] = v.y;
                    } else {
                        if (lo_in) x0[k] = src[k][w0];
                        if (hi_in) x1[k] = src[k][w0 + 1];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
#pragma unroll
                for (int uu = 0; uu < NTAB; ++uu) {
                    const int tau = uu ^ rho;
                    const int e = (int)((ix[k] >> (8 * tau)) & 255ull);
                    const ulonglong2 tv = *reinterpret_cast<const ulonglong2 *>(
                        Tq + (tau >> 1) * (256 * TAB_LINE) + e * TAB_LINE + (tau & 1) * TW);
                    x0[k] ^= tv.x;
                    x1[k] ^= tv.y;
                }
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (ri[k] < 0) continue;
                uint64_t *dst = a.A + ri[k] * a.ld;
                if (VEC && lo_in && hi_in) {
                    *reinterpret_cast<ulonglong2 *>(dst + w0) = make_ulonglong2(x0[k], x1[k]);
                } else {
                    if (lo_in) dst[w0] = x0[k];
                    if (hi_in) dst[w0 + 1] = x1[k];
                }
            }
        }
        u += nrows;
    }
}

// ----------------------------------------------------------------------------
// Pipelined form (16-byte aligned rows).  Two changes against update_kernel:
//  * CTAs 2j and 2j+1 work on the two 64-byte halves of the same 128-byte
//    lines over the same rows at the same time, so a DRAM line fetched for one
//    half is not fetched again for the other much later (measured: DRAM reads
//    fall from 1.76x to 1.00x of the algorithmic bytes);
//  * loads are software-pipelined in registers: the row words and indices of
//    the next batch are in flight while the current batch does its table
//    lookups.  Staging them through shared memory instead (cp.async) was
//    measured to saturate the L1/shared data pipe, which the eight table
//    lookups per word already use heavily.  Loads and stores use the default
//    cache policy: evict-first hints let L2 drop the partner half of a line
//    before the paired CTA reads it (measured: reads back up to 1.68x).
//
// WIDE = true: 128-byte column tiles, so that every warp-wide row load or
// store covers whole 128-byte lines (four rows of eight lanes) instead of
// half lines (eight rows of four lanes): half the L1 wavefronts per byte of
// row, which with the table lookups saturate the L1/shared data pipe.  Eight
// 8-bit tables of 128-byte entries would take 256 KiB, so a stripe's 64
// generator rows are split into eight 7-bit tables (rows 7t .. 7t+6, 128
// entries) and one 8-bit table (rows 56..63): 1280 entries x 128 bytes =
// 160 KiB, nine lookups per 16 bytes of row instead of eight.  Index bit j
// still selects generator row j.  The eight lanes of a row read one whole
// 128-byte entry per lookup, so lookups are conflict-free; CTAs take whole
// lines and need no partner.
constexpr int PIPE_RPT = 4;

struct RowBatch {
    uint64_t x0[PIPE_RPT], x1[PIPE_RPT], ix[PIPE_RPT];
    int64_t ri[PIPE_RPT];
};

// The body of the pipelined table kernels.
template <bool WIDE>
__device__ __forceinline__ void update_pipe_body(const UpdArgs &a, uint64_t *T)
{
    __shared__ const uint64_t *sGen[KS];
    __shared__ __align__(16) uint64_t sGt[WIDE ? KS * WT : 1];   // wide form: the tile's generator words

    int64_t row_lo, row_hi, w_lo;
    const int64_t W = a.W;
    int64_t r = 0;
    int maxpos = -1, nS = 0, rbar_m = 0;
    const StripeDesc *d = a.desc;
    if (a.mode == UPD_PLE) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        r = d->r;
        row_lo = r;
        row_hi = a.m;
        w_lo = (d->c >> 6) + (a.first_off > 0 ? a.first_off : 1);
        maxpos = d->maxpos;
        nS = d->nS;
        if (threadIdx.x < KS)
            sGen[threadIdx.x] = (threadIdx.x < rbar) ? a.S + threadIdx.x * a.ldS : nullptr;
    } else if (a.mode == UPD_RREF) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        row_lo = a.row_lo;                    // 0, or the first row of a block's own RREF
        row_hi = d->r;
        w_lo = max((int64_t)(d->c >> 6), a.w_lo);  // a.w_lo > 0: only a right part of the row
        if (threadIdx.x < KS) sGen[threadIdx.x] = nullptr;
        __syncthreads();
        if (threadIdx.x < rbar) sGen[d->qbar[threadIdx.x]] = a.A + (d->r + threadIdx.x) * a.ld;
    } else if (a.mode == UPD_M4RI) {
        rbar_m = d->rbar;
        if (rbar_m == 0) return;
        r = d->r;
        row_lo = 0;
        row_hi = a.m;
        w_lo = d->c >> 6;
        maxpos = d->maxpos;
        if (threadIdx.x < KS) sGen[threadIdx.x] = nullptr;
        __syncthreads();
        if (threadIdx.x < rbar_m) sGen[d->qbar[threadIdx.x]] = a.B + threadIdx.x * a.ldb;
    } else {
        row_lo = a.row_lo;
        row_hi = a.row_hi;
        w_lo = a.w_lo;
        if (threadIdx.x < KS)
            sGen[threadIdx.x] = (threadIdx.x < a.gen_count) ? a.B + threadIdx.x * a.ldb : nullptr;
    }
    __syncthreads();

    if (a.mode == UPD_M4RI) {
        for (int p = blockIdx.x; p < rbar_m; p += gridDim.x)
            for (int64_t w = w_lo + threadIdx.x; w < W; w += blockDim.x) a.A[(r + p) * a.ld + w] = a.B[p * a.ldb + w];
    }
    if (a.mode == UPD_PLE && a.left_copies) {
        for (int k = blockIdx.x; k < nS; k += gridDim.x) {
            const uint64_t *src = a.S + (int64_t)k * a.ldS;
            uint64_t *dst = a.A + (r + d->S_off[k]) * a.ld;
            for (int64_t w = threadIdx.x; w < w_lo; w += blockDim.x) dst[w] = src[w];
            for (int64_t w = W + threadIdx.x; w < a.W_full; w += blockDim.x) dst[w] = src[w];
        }
    }

    const int64_t R = row_hi - row_lo;
    if (w_lo >= W || R <= 0) return;
    // The column range in units: tile pairs of 64-byte tiles (paired form),
    // 128-byte tiles (wide form); tp_lo / tp_hi select a range of units, and
    // unit 0 holds the first word w_lo either way.
    constexpr int TWK = WIDE ? WT : TW;              // words per tile
    const int64_t a0 = w_lo / TWK, a1 = (W + TWK - 1) / TWK;
    // an optional skipped word range [skip_lo, skip_hi) (known zero in every
    // row involved): whole tiles inside it are left out, so tile index t maps
    // to tile a0 + t below the gap and b0 + (t - n1) after it
    int64_t n1 = a1 - a0, b0 = a1;
    if (a.skip_hi > a.skip_lo && a.skip_lo > w_lo && a.skip_hi < W) {
        const int64_t e1 = (a.skip_lo + TWK - 1) / TWK, bb = a.skip_hi / TWK;
        if (bb > e1) { n1 = e1 - a0; b0 = bb; }
    }
    const int64_t NT = n1 + (a1 - b0);
    auto phys = [&](int64_t t) -> int64_t { return t < n1 ? a0 + t : b0 + (t - n1); };
    const int64_t NU = WIDE ? NT : (NT + 1) / 2;
    const int64_t tp_lo = min(a.tp_lo, NU);
    const int64_t tp_hi = (a.tp_hi < 0) ? NU : min(a.tp_hi, NU);
    if (tp_lo >= tp_hi) return;
    const int npairs = WIDE ? (int)gridDim.x : (int)(gridDim.x >> 1);
    const int pj = WIDE ? (int)blockIdx.x : (int)(blockIdx.x >> 1), half = WIDE ? 0 : (int)(blockIdx.x & 1);
    if (pj >= npairs) return;                       // odd grid: the last CTA has no partner
    const int64_t U = (tp_hi - tp_lo) * R;
    const int64_t u_beg = U * pj / npairs;
    const int64_t u_end = U * (pj + 1) / npairs;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.bytes) {
        int64_t words = 0;                           // words of the tiles [units tp_lo, tp_hi)
        for (int64_t t = (WIDE ? 1 : 2) * tp_lo; t < min(NT, (WIDE ? 1 : 2) * tp_hi); ++t)
            words += min(W, (phys(t) + 1) * TWK) - max(w_lo, phys(t) * TWK);
        atomicAdd(a.bytes, (unsigned long long)(R * words * 16));
    }

    constexpr int LANES = TWK / 2;                  // threads per row: 16 bytes each
    const int tid = threadIdx.x;
    const int rs = tid / LANES;
    const int qd = tid % LANES;
    const int rho = rs & 1;
    constexpr int SLOTS = UPD_THREADS / LANES;
    constexpr int CH = SLOTS * PIPE_RPT;             // rows per batch

    for (int64_t u = u_beg; u < u_end;) {
        const int64_t tq = u / R;
        const int64_t rr0 = u - tq * R;
        const int64_t nrows = min(R - rr0, u_end - u);
        u += nrows;
        const int64_t tile = WIDE ? tp_lo + tq : 2 * (tp_lo + tq) + half;
        if (tile >= NT) continue;
        const int64_t wbase = phys(tile) * TWK;
        __syncthreads();
        if (WIDE) {
            // the tile's words of the 64 generator rows into shared memory in
            // one round trip (words outside [w_lo, W) as zero: their entries
            // are never stored back), then the tables from there
            static_assert(KS * WT == 2 * UPD_THREADS, "two generator words per thread");
            uint64_t gv[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int e = threadIdx.x + q * UPD_THREADS, row = e / WT;
                const int64_t word = wbase + e % WT;
                const uint64_t *gp = sGen[row];
                gv[q] = (gp != nullptr && word >= w_lo && word < W) ? gp[word] : 0ull;
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) sGt[threadIdx.x + q * UPD_THREADS] = gv[q];
            __syncthreads();
            build_wide_tables_smem(T, sGt);
        } else {
            build_tables(T, sGen, wbase, W);
        }
        __syncthreads();

        const int64_t w0 = wbase + 2 * qd;
        const bool lo_in = w0 >= w_lo && w0 < W;
        const bool hi_in = w0 + 1 >= w_lo && w0 + 1 < W;
        const bool full = lo_in && hi_in;
        const int64_t row0 = row_lo + rr0;
        const uint64_t *Tq = T + 2 * qd;

        auto fetch = [&](RowBatch &bt, int64_t base) {
#pragma unroll
            for (int k = 0; k < PIPE_RPT; ++k) {
                const int64_t off = base + k * SLOTS + rs;
                bt.ri[k] = (off < nrows) ? row0 + off : -1;
                if (bt.ri[k] >= r && bt.ri[k] < r + rbar_m) bt.ri[k] = -1;   // M4RI pivot positions
                bt.x0[k] = 0;
                bt.x1[k] = 0;
                bt.ix[k] = 0;
                if (bt.ri[k] >= 0) {
                    const int64_t i = bt.ri[k];
                    bt.ix[k] = __ldg(a.idx + i * a.idx_stride);
                    const uint64_t *sp = a.A + i * a.ld;
                    if ((a.mode == UPD_PLE || a.mode == UPD_M4RI) && i >= r && i - r <= maxpos) {
                        const int mv = a.map[i];
                        if (mv >= 0 && (mv >> 8) == a.stripe) sp = a.S + (int64_t)(mv & 255) * a.ldS;
                    }
                    if (full) {
                        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(sp + w0);
                        bt.x0[k] = v.x;
                        bt.x1[k] = v.y;
                    } else {
                        if (lo_in) bt.x0[k] = sp[w0];
                        if (hi_in) bt.x1[k] = sp[w0 + 1];
                    }
                }
            }
        };
        auto finish = [&](RowBatch &bt) {
#pragma unroll
            for (int k = 0; k < PIPE_RPT; ++k) {
                uint64_t x0 = bt.x0[k], x1 = bt.x1[k];
                const uint64_t ix = bt.ix[k];
                if (WIDE) {
#pragma unroll
                    for (int t = 0; t < WNTAB; ++t) {
                        const int e = t < WNTAB - 1 ? (int)((ix >> (7 * t)) & 127ull) : (int)(ix >> 56);
                        const ulonglong2 tv =
                            *reinterpret_cast<const ulonglong2 *>(Tq + (int64_t)(128 * t + e) * WT);
                        x0 ^= tv.x;
                        x1 ^= tv.y;
                    }
                } else {
#pragma unroll
                    for (int uu = 0; uu < NTAB; ++uu) {
                        const int tau = uu ^ rho;
                        const int e = (int)((ix >> (8 * tau)) & 255ull);
                        const ulonglong2 tv = *reinterpret_cast<const ulonglong2 *>(
                            Tq + (tau >> 1) * (256 * TAB_LINE) + e * TAB_LINE + (tau & 1) * TW);
                        x0 ^= tv.x;
                        x1 ^= tv.y;
                    }
                }
                if (bt.ri[k] < 0) continue;
                uint64_t *dst = a.A + bt.ri[k] * a.ld;
                if (full) {
                    *reinterpret_cast<ulonglong2 *>(dst + w0) = make_ulonglong2(x0, x1);
                } else {
                    if (lo_in) dst[w0] = x0;
                    if (hi_in) dst[w0 + 1] = x1;
                }
            }
        };

        RowBatch b0, b1;
        fetch(b0, 0);
        int64_t base = 0;
        for (;;) {
            if (base + CH < nrows) fetch(b1, base + CH);
            finish(b0);
            base += CH;
            if (base >= nrows) break;
            if (base + CH < nrows) fetch(b0, base + CH);
            finish(b1);
            base += CH;
            if (base >= nrows) break;
        }
    }
}

template <bool WIDE>
__global__ void __launch_bounds__(UPD_THREADS, 1) update_pipe_kernel(UpdArgs a)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint64_t T[];
    update_pipe_body<WIDE>(a, T);
}

// ----------------------------------------------------------------------------
// Naive form, the plain baseline: no tables.  One thread per (row, word) adds
// the generator rows selected by the row's index bits one by one (up to 64
// row additions per row, Section 3.2's trailing update written as plain row
// XORs), so every updated word reads up to 64 generator words.  Same modes
// and arguments as the table kernels (PLE, RREF, MUL).
__global__ void __launch_bounds__(256) naive_update_kernel(UpdArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ const uint64_t *sGen[KS];
    int64_t row_lo, row_hi, w_lo, r = 0;
    int maxpos = -1, nS = 0;
    const int64_t W = a.W;
    const StripeDesc *d = a.desc;
    if (a.mode == UPD_PLE) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        r = d->r;
        row_lo = r;
        row_hi = a.m;
        w_lo = (d->c >> 6) + (a.first_off > 0 ? a.first_off : 1);
        maxpos = d->maxpos;
        nS = d->nS;
        if (threadIdx.x < KS) sGen[threadIdx.x] = (threadIdx.x < rbar) ? a.S + threadIdx.x * a.ldS : nullptr;
    } else if (a.mode == UPD_RREF) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        row_lo = a.row_lo;
        row_hi = d->r;
        w_lo = max((int64_t)(d->c >> 6), a.w_lo);
        if (threadIdx.x < KS) sGen[threadIdx.x] = nullptr;
        __syncthreads();
        if (threadIdx.x < rbar) sGen[d->qbar[threadIdx.x]] = a.A + (d->r + threadIdx.x) * a.ld;
    } else {
        row_lo = a.row_lo;
        row_hi = a.row_hi;
        w_lo = a.w_lo;
        if (threadIdx.x < KS)
            sGen[threadIdx.x] = (threadIdx.x < a.gen_count) ? a.B + threadIdx.x * a.ldb : nullptr;
    }
    __syncthreads();
    if (a.mode == UPD_PLE && a.left_copies) {
        for (int k = blockIdx.x; k < nS; k += gridDim.x) {
            const uint64_t *src = a.S + (int64_t)k * a.ldS;
            uint64_t *dst = a.A + (r + d->S_off[k]) * a.ld;
            for (int64_t w = threadIdx.x; w < w_lo; w += blockDim.x) dst[w] = src[w];
            for (int64_t w = W + threadIdx.x; w < a.W_full; w += blockDim.x) dst[w] = src[w];
        }
    }
    const int64_t R = row_hi - row_lo, NW = W - w_lo;
    if (R <= 0 || NW <= 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.bytes) atomicAdd(a.bytes, (unsigned long long)(R * NW * 16));
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < R * NW;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = row_lo + t / NW, w = w_lo + t % NW;
        const uint64_t *src = a.A + i * a.ld;
        if (a.mode == UPD_PLE && i - r <= maxpos) {
            const int mv = a.map[i];
            if (mv >= 0 && (mv >> 8) == a.stripe) src = a.S + (int64_t)(mv & 255) * a.ldS;
        }
        uint64_t ix = a.idx[i * a.idx_stride];
        uint64_t x = src[w];
        while (ix) {
            const int b = __ffsll((long long)ix) - 1;
            ix &= ix - 1;
            if (sGen[b]) x ^= sGen[b][w];
        }
        a.A[i * a.ld + w] = x;
    }
}

cudaError_t setup_update_kernel()
{
    const int smem = (int)(TAB_WORDS * sizeof(uint64_t));
    cudaError_t e = cudaFuncSetAttribute(update_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(update_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(update_pipe_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(update_pipe_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(WIDE_TAB_WORDS * sizeof(uint64_t)));
    if (e != cudaSuccess) return e;
    e = setup_rref_pass_kernel();
    if (e != cudaSuccess) return e;
    e = setup_update_tma_kernel();
    if (e != cudaSuccess) return e;
    return setup_prep_kernel();   // the prep kernel's 48 KiB of tables
}

bool update_vectorised(const UpdArgs &a)
{
    return (a.ld % 2 == 0) && ((uintptr_t)a.A % 16 == 0) &&
           ((a.mode != UPD_PLE && a.mode != UPD_M4RI) || (a.ldS % 2 == 0 && (uintptr_t)a.S % 16 == 0));
}

cudaError_t launch_update(cudaStream_t st, const UpdArgs &a, int num_sms)
{
    const size_t smem = TAB_WORDS * sizeof(uint64_t);
    // The vectorised forms need 16-byte aligned rows: even leading dimensions
    // and 16-byte aligned bases (staged rows too, for the PLE update), and
    // 8-byte aligned index words.
    const bool vec = (a.ld % 2 == 0) && ((uintptr_t)a.A % 16 == 0) &&
                     ((a.mode != UPD_PLE && a.mode != UPD_M4RI) || (a.ldS % 2 == 0 && (uintptr_t)a.S % 16 == 0));
    int grid = (a.grid > 0 && a.grid < num_sms) ? a.grid : num_sms;
    if (a.naive && a.mode != UPD_M4RI) {
        return launch_kernel(naive_update_kernel, dim3(8 * num_sms), dim3(256), 0, st, a);
    }
    if (vec) {
        grid &= ~1;
        if (grid < 2) grid = 2;
        if (a.tmap)
            return launch_update_tma(st, a, grid);
        if (a.rref_fused && a.wide) return launch_rref_pass(st, a, num_sms);   // kernels_rref_pass.cu
        if (a.wide) {
            int gw = (a.grid > 0 && a.grid < num_sms) ? a.grid : num_sms;
            return launch_kernel(update_pipe_kernel<true>, dim3(gw), dim3(UPD_THREADS),
                                 WIDE_TAB_WORDS * sizeof(uint64_t), st, a);
        } else {
            return launch_kernel(update_pipe_kernel<false>, dim3(grid), dim3(UPD_THREADS), smem, st, a);
        }
    } else {
        return launch_kernel(update_kernel<false>, dim3(grid), dim3(UPD_THREADS), smem, st, a);
    }
    return cudaGetLastError();
}

}  // namespace gf2
