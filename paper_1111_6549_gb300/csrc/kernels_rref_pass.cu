// kernels_rref_pass.cu -- one stripe pass of the blocked RREF recovery's base
// blocks, with the stripe's block reduction fused in (Section 5's RREF, read
// as back-substitution by pivot blocks).
//
// Pass s clears the pivot columns of stripe s from the rows [row_lo, r_s)
// above the stripe, over the words [c_s / 64, W) less a skipped range known
// to be zero there.  Each row above takes the XOR of the stripe's reduced
// pivot rows G = U11^-1 (raw pivot rows) selected by its bits on the pivot
// columns (its stripe word, snapshotted by the previous pass).  Per 128-byte
// column tile a CTA
//   1. loads the tile of the raw pivot rows and the first batch of its rows
//      above; both are in flight while the pass's side jobs run;
//   2. forms G on the tile by the Four Russians method applied to U11^-1:
//      sixteen 16-entry tables of combinations of four raw rows each, then
//      sixteen lookups per word of G, one per 4-bit field of the row of
//      U11^-1 (instead of 64 masked XORs);
//   3. puts G, by pivot column, into the nine update tables (160 KiB) and
//      into a buffer from which the next pass writes it back to the pivot
//      rows, once no CTA reads them raw any more;
//   4. updates its rows above on the tile: nine table lookups per 16 bytes.
// Side jobs (grid-stride over every CTA): the previous pass's write-back and
// the next pass's index snapshot.
#include "common.cuh"
#include "tables_dev.cuh"

namespace gf2 {

namespace {

constexpr int RP_RPT = 4;                 // rows per thread and batch
constexpr int RP_LANES = WT / 2;          // threads per row: 16 bytes each
constexpr int RP_SLOTS = UPD_THREADS / RP_LANES;
constexpr int RP_CH = RP_SLOTS * RP_RPT;  // rows per batch
constexpr int RP_GROUPS = KS / 4;         // 4-row groups of the raw pivot rows

struct RpBatch {
    uint64_t x0[RP_RPT], x1[RP_RPT], ix[RP_RPT];
    int64_t ri[RP_RPT];
};

// The fused pass's bookends: the previous pass's reduced pivot rows from
// gbuf_r into A, and the next pass's table index.  Neither touches a word
// this pass reads or writes: the previous stripe's pivot rows lie below this
// stripe's rows, and the next stripe's word lies left of this pass's words.
__device__ __forceinline__ void rref_side_jobs(const UpdArgs &a, int64_t W)
{
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    if (a.flush_desc) {
        const StripeDesc *f = a.flush_desc;
        const int rbar = f->rbar;
        const int64_t c0 = f->c >> 6;
        const int64_t nw = W - c0;
        if (rbar > 0 && nw > 0)
            for (int64_t e = gt; e < rbar * nw; e += gs) {
                const int64_t t = e / nw, word = c0 + (e - t * nw);
                if (word >= a.skip_lo && word < a.skip_hi) continue;
                a.A[(f->r + t) * a.ld + word] = a.gbuf_r[t * a.ldg + word];
            }
    }
    if (a.snap_desc) {
        const StripeDesc *sd = a.snap_desc;
        const int64_t cw = sd->c >> 6;
        for (int64_t i = a.row_lo + gt; i < sd->r; i += gs) a.idx_next[i] = a.A[i * a.ld + cw];
    }
}

}  // namespace

__global__ void __launch_bounds__(UPD_THREADS, 1) rref_pass_kernel(UpdArgs a)
{
    pdl_wait();
    pdl_trigger();
    // the nine update tables; before they are built, the tile of the raw
    // pivot rows and its 4-row combinations live in the same space
    extern __shared__ __align__(16) uint64_t T[];
    uint64_t *sRaw = T;                                  // [pivot row][tile word]
    uint64_t *sC = T + KS * WT;                          // [group][combination][tile word]
    __shared__ __align__(16) uint64_t sGc[KS * WT];      // G by pivot column
    __shared__ uint64_t sMinv[KS];
    __shared__ int8_t sCol[KS];

    const int tid = threadIdx.x;
    const StripeDesc *d = a.desc;
    const int64_t W = a.W;
    const int rbar = d->rbar;
    const int64_t rp = d->r;                             // first pivot row; the rows above end here
    const int64_t row_lo = a.row_lo;
    const int64_t R = rp - row_lo;
    const int64_t w_lo = max((int64_t)(d->c >> 6), a.w_lo);
    if (tid < KS) {
        sMinv[tid] = tid < rbar ? d->Minv[tid] : 0ull;
        sCol[tid] = tid < rbar ? (int8_t)d->qbar[tid] : (int8_t)-1;
    }
    // the column tiles: whole tiles inside the skipped range are left out,
    // so tile t maps to a0 + t below the gap and b0 + (t - n1) after it
    const int64_t a0 = w_lo / WT, a1 = (W + WT - 1) / WT;
    int64_t n1 = a1 - a0, b0 = a1;
    if (a.skip_hi > a.skip_lo && a.skip_lo > w_lo && a.skip_hi < W) {
        const int64_t e1 = (a.skip_lo + WT - 1) / WT, bb = a.skip_hi / WT;
        if (bb > e1) { n1 = e1 - a0; b0 = bb; }
    }
    const int64_t NT = (rbar > 0 && w_lo < W) ? n1 + (a1 - b0) : 0;
    auto phys = [&](int64_t t) -> int64_t { return t < n1 ? a0 + t : b0 + (t - n1); };
    // units: (tile, row) pairs, tile-major; with no rows above, one unit per tile
    const int64_t Ru = R > 0 ? R : 1;
    const int64_t U = NT * Ru;
    const int64_t u_beg = U * blockIdx.x / gridDim.x, u_end = U * (blockIdx.x + 1) / gridDim.x;
    if (blockIdx.x == 0 && tid == 0 && a.bytes && R > 0) {
        int64_t words = 0;
        for (int64_t t = 0; t < NT; ++t) words += min(W, (phys(t) + 1) * WT) - max(w_lo, phys(t) * WT);
        atomicAdd(a.bytes, (unsigned long long)(R * words * 16));
    }

    const int rs = tid / RP_LANES, qd = tid % RP_LANES;
    // the current tile
    int64_t wbase = 0, row0 = 0, nrows = 0, w0 = 0;
    bool lo_in = false, hi_in = false, full = false;
    auto set_tile = [&](int64_t u) {
        const int64_t tq = u / Ru, rr0 = u - tq * Ru;
        nrows = R > 0 ? min(R - rr0, u_end - u) : 0;
        wbase = phys(tq) * WT;
        row0 = row_lo + rr0;
        w0 = wbase + 2 * qd;
        lo_in = w0 >= w_lo && w0 < W;
        hi_in = w0 + 1 >= w_lo && w0 + 1 < W;
        full = lo_in && hi_in;
    };
    uint64_t raw[2];
    auto load_raw = [&]() {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = tid + h * UPD_THREADS, t = e / WT;
            const int64_t word = wbase + e % WT;
            raw[h] = (t < rbar && word < W) ? a.A[(rp + t) * a.ld + word] : 0ull;
        }
    };
    auto fetch = [&](RpBatch &bt, int64_t base) {
#pragma unroll
        for (int k = 0; k < RP_RPT; ++k) {
            const int64_t off = base + k * RP_SLOTS + rs;
            bt.ri[k] = (off < nrows) ? row0 + off : -1;
            bt.x0[k] = 0;
            bt.x1[k] = 0;
            bt.ix[k] = 0;
            if (bt.ri[k] >= 0) {
                const int64_t i = bt.ri[k];
                bt.ix[k] = __ldg(a.idx + i * a.idx_stride);
                const uint64_t *sp = a.A + i * a.ld;
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
    auto finish = [&](RpBatch &bt) {
        const uint64_t *Tq = T + 2 * qd;
#pragma unroll
        for (int k = 0; k < RP_RPT; ++k) {
            uint64_t x0 = bt.x0[k], x1 = bt.x1[k];
            const uint64_t ix = bt.ix[k];
#pragma unroll
            for (int t = 0; t < WNTAB; ++t) {
                const int e = t < WNTAB - 1 ? (int)((ix >> (7 * t)) & 127ull) : (int)(ix >> 56);
                const ulonglong2 tv = *reinterpret_cast<const ulonglong2 *>(Tq + (int64_t)(128 * t + e) * WT);
                x0 ^= tv.x;
                x1 ^= tv.y;
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

    // the first tile's loads go out before the side jobs
    RpBatch bA, bB;
    int64_t u = u_beg;
    if (u < u_end) {
        set_tile(u);
        load_raw();
        fetch(bA, 0);
    }
    rref_side_jobs(a, W);
    bool first = true;
    while (u < u_end) {
        if (!first) {
            set_tile(u);
            load_raw();
            fetch(bA, 0);
        }
        first = false;
        u += nrows > 0 ? nrows : 1;
        __syncthreads();                                 // the previous tile's tables are no longer read
        sRaw[tid] = raw[0];
        sRaw[tid + UPD_THREADS] = raw[1];
        for (int e = tid; e < KS * WT; e += UPD_THREADS) sGc[e] = 0ull;
        __syncthreads();
        // combinations of the raw rows 4g .. 4g+3, word by word: thread
        // (pair p, half h) forms combinations 8h .. 8h+7 of pair p = (g, word)
        {
            const int p = tid & 255, h = tid >> 8;
            const int g = p / WT, ww = p % WT;
            const uint64_t r0 = sRaw[(4 * g) * WT + ww], r1 = sRaw[(4 * g + 1) * WT + ww];
            const uint64_t r2 = sRaw[(4 * g + 2) * WT + ww], r3 = sRaw[(4 * g + 3) * WT + ww];
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) {
                const int c = 8 * h + c8;
                sC[(16 * g + c) * WT + ww] = ((c & 1) ? r0 : 0ull) ^ ((c & 2) ? r1 : 0ull) ^ ((c & 4) ? r2 : 0ull) ^
                                             ((c & 8) ? r3 : 0ull);
            }
        }
        __syncthreads();
        // G = U11^-1 (raw rows): one lookup per 4-bit field of the row of U11^-1
        for (int e = tid; e < KS * WT; e += UPD_THREADS) {
            const int t = e / WT, ww = e % WT;
            if (t >= rbar) continue;
            const uint64_t mrow = sMinv[t];
            uint64_t acc = 0;
#pragma unroll
            for (int g = 0; g < RP_GROUPS; ++g) acc ^= sC[(16 * g + (int)((mrow >> (4 * g)) & 15ull)) * WT + ww];
            sGc[sCol[t] * WT + ww] = acc;
            const int64_t word = wbase + ww;
            const bool in_skip = word >= a.skip_lo && word < a.skip_hi;
            if (word >= w_lo && word < W && !in_skip) a.gbuf_w[t * a.ldg + word] = acc;
        }
        __syncthreads();
        build_wide_tables_smem(T, sGc);
        __syncthreads();
        if (nrows <= 0) continue;
        int64_t base = 0;
        for (;;) {
            if (base + RP_CH < nrows) fetch(bB, base + RP_CH);
            finish(bA);
            base += RP_CH;
            if (base >= nrows) break;
            if (base + RP_CH < nrows) fetch(bA, base + RP_CH);
            finish(bB);
            base += RP_CH;
            if (base >= nrows) break;
        }
    }
}

cudaError_t setup_rref_pass_kernel()
{
    return cudaFuncSetAttribute(rref_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(WIDE_TAB_WORDS * sizeof(uint64_t)));
}

cudaError_t launch_rref_pass(cudaStream_t st, const UpdArgs &a, int num_sms)
{
    const int grid = (a.grid > 0 && a.grid < num_sms) ? a.grid : num_sms;
    return launch_kernel(rref_pass_kernel, dim3(grid), dim3(UPD_THREADS), WIDE_TAB_WORDS * sizeof(uint64_t), st, a);
}

}  // namespace gf2
