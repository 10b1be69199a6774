// kernels_batched.cu -- many independent PLE decompositions in one persistent
// launch.
//
// Every CTA claims whole matrices from an atomic work counter over a list
// sorted largest first, and runs the complete block-iterative PLE
// (Algorithm 2) of each claimed matrix by itself: per 64-column stripe the
// pivot search of Algorithm 1 (panel_dev.cuh: the warp window, else the
// block-wide path), the L bits and table indices of every row, and the
// tabulated update of the columns right of the stripe.  The matrices of the
// batched workload (64..1024 rows and columns) stay in L2 while their CTA
// works on them, and no CTA ever waits for another, so the kernel has no
// cross-CTA synchronisation at all.
#include "panel_dev.cuh"

namespace gf2 {

constexpr int BATCH_THREADS = 256;
constexpr int BTW = 2;                               // table tile: 2 words (16 bytes) per row
constexpr int BTAB_WORDS = NTAB * 256 * BTW;         // 32 KiB of tables

struct BatchScratch {
    uint64_t *idx;       // per CTA: max_rows words
    uint64_t *S;         // per CTA: SMAX staged rows of ldS words
    uint64_t *gval;      // per CTA: block-wide panel scratch
    uint64_t *glb;
    int32_t *gsrc;
    int64_t max_rows, ldS;
};

__device__ __forceinline__ void batch_write_lregion(uint64_t *row, int64_t r, int64_t cw, int rbar,
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

__global__ void __launch_bounds__(BATCH_THREADS, 4)
batched_ple_kernel(const gf2_batch_item *items, const int32_t *order, int count, int32_t *next,
                   BatchScratch scr)
{
    extern __shared__ __align__(16) uint64_t T[];    // BTAB_WORDS: [table][entry][BTW]
    __shared__ PanelShared sh;
    __shared__ uint64_t sLinv[KS];
    __shared__ int16_t smap[BATCH_MAX_ROWS];          // position offset -> staged slot, or -1
    __shared__ int sh_item;
    __shared__ uint64_t sG[KS * BTW];                 // generator words of the current tile

    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t *idx = scr.idx + (size_t)blockIdx.x * scr.max_rows;
    uint64_t *S = scr.S + (size_t)blockIdx.x * SMAX * scr.ldS;
    PanelScratch gs{scr.gval + (size_t)blockIdx.x * scr.max_rows, scr.glb + (size_t)blockIdx.x * scr.max_rows,
                    scr.gsrc + (size_t)blockIdx.x * scr.max_rows};
    const int64_t ldS = scr.ldS;

    for (;;) {
        __syncthreads();
        if (tid == 0) sh_item = atomicAdd(next, 1);
        __syncthreads();
        const int b = sh_item;
        if (b >= count) break;
        const gf2_batch_item it = items[order[b]];
        uint64_t *A = it.A;
        const int64_t m = it.m, n = it.n, ld = it.ld_words;
        const int64_t qn = m < n ? m : n;
        for (int64_t i = tid; i < m; i += BATCH_THREADS) {
            it.P[i] = i;
            if (i < qn) it.Q[i] = -1;
            smap[i] = -1;
        }
        __syncthreads();
        const int64_t W = (n + 63) >> 6;
        int64_t r = 0;
        for (int64_t s = 0; s < W && r < m; ++s) {
            __syncthreads();                      // everyone is done with the last stripe's sh
            const int64_t c = s * KS, cw = s;
            const int keff = (int)min((int64_t)KS, n - c);
            const int64_t rows = m - r;
            if (warp == 0) panel_window(A, r, ld, cw, rows, keff, sh);
            __syncthreads();
            if (sh.fail) panel_block(A, r, ld, cw, rows, keff, gs, sh, nullptr);
            __syncthreads();
            const int rbar = sh.rbar;
            if (rbar == 0) continue;
            if (warp == 0) warp_lower_inverse(sh.L, rbar, sLinv);
            for (int p = tid; p < rbar; p += BATCH_THREADS) {
                it.P[r + p] = r + sh.t[p];
                it.Q[r + p] = c + sh.j[p];
            }
            const int nS = sh.nS;
            const int maxpos = sh.maxpos;
            for (int k = tid; k < nS; k += BATCH_THREADS) smap[sh.Soff[k]] = (int16_t)k;
            for (int64_t t = tid; t < (int64_t)nS * W; t += BATCH_THREADS) {
                const int64_t k = t / W, w = t - k * W;
                S[k * ldS + w] = A[sh.Ssrc[k] * ld + w];
            }
            __syncthreads();
            // every row at a position >= r: L bits in place (staged rows: in S)
            // and the table index
            for (int64_t off = tid; off < rows; off += BATCH_THREADS) {
                const int k = (off <= maxpos) ? smap[off] : -1;
                uint64_t *row = (k >= 0) ? S + (int64_t)k * ldS : A + (r + off) * ld;
                uint64_t v, es = 0, ix = 0;
                if (k >= 0 && k < rbar) {
                    v = sh.L[k];
                    es = sh.E[k];
                    ix = sLinv[k] ^ (1ull << k);
                } else {
                    uint64_t sw = row[cw];
                    v = 0;
                    for (int p = 0; p < rbar; ++p) {
                        const uint64_t bit = (sw >> sh.j[p]) & 1ull;
                        sw ^= sh.E[p] & (0ull - bit);
                        v |= bit << p;
                    }
                    for (int p = 0; p < rbar; ++p) ix ^= sLinv[p] & (0ull - ((v >> p) & 1ull));
                }
                batch_write_lregion(row, r, cw, rbar, v, es);
                idx[off] = ix;
            }
            __syncthreads();
            // tabulated update of the words right of the stripe
            const int64_t w_lo = cw + 1;
            for (int64_t wbase = (w_lo / BTW) * BTW; wbase < W; wbase += BTW) {
                // T[tau][e][x] = XOR of generator rows 8 tau + bit of e, word wbase + x
                for (int t = tid; t < KS * BTW; t += BATCH_THREADS) {
                    const int g = t / BTW, x = t - g * BTW;
                    sG[t] = (g < rbar && wbase + x < W) ? S[(int64_t)g * ldS + wbase + x] : 0ull;
                }
                __syncthreads();
                for (int e2 = tid; e2 < NTAB * 256; e2 += BATCH_THREADS) {
                    const int tau = e2 >> 8, e = e2 & 255;
                    uint64_t acc[BTW];
#pragma unroll
                    for (int x = 0; x < BTW; ++x) acc[x] = 0;
#pragma unroll
                    for (int bq = 0; bq < 8; ++bq) {
                        const uint64_t msk = 0ull - (uint64_t)((e >> bq) & 1);
#pragma unroll
                        for (int x = 0; x < BTW; ++x) acc[x] ^= sG[(8 * tau + bq) * BTW + x] & msk;
                    }
#pragma unroll
                    for (int x = 0; x < BTW; ++x) T[(size_t)e2 * BTW + x] = acc[x];
                }
                __syncthreads();
                for (int64_t off = tid; off < rows; off += BATCH_THREADS) {
                    const int k = (off <= maxpos) ? smap[off] : -1;
                    const uint64_t *src = (k >= 0) ? S + (int64_t)k * ldS : A + (r + off) * ld;
                    uint64_t *dst = A + (r + off) * ld;
                    const uint64_t ix = idx[off];
                    uint64_t acc[BTW];
#pragma unroll
                    for (int x = 0; x < BTW; ++x) {
                        const int64_t w = wbase + x;
                        acc[x] = (w >= w_lo && w < W) ? src[w] : 0ull;
                    }
#pragma unroll
                    for (int tau = 0; tau < NTAB; ++tau) {
                        const int e = (int)((ix >> (8 * tau)) & 255ull);
                        const uint64_t *te = T + ((size_t)tau * 256 + e) * BTW;
#pragma unroll
                        for (int x = 0; x < BTW; ++x) acc[x] ^= te[x];
                    }
#pragma unroll
                    for (int x = 0; x < BTW; ++x) {
                        const int64_t w = wbase + x;
                        if (w >= w_lo && w < W) dst[w] = acc[x];
                    }
                }
                __syncthreads();
            }
            // staged rows: their left part (old L bits, new L bits, stripe)
            for (int64_t t = tid; t < (int64_t)nS * (cw + 1); t += BATCH_THREADS) {
                const int64_t k = t / (cw + 1), w = t - k * (cw + 1);
                A[(r + sh.Soff[k]) * ld + w] = S[k * ldS + w];
            }
            __syncthreads();
            for (int k = tid; k < nS; k += BATCH_THREADS) smap[sh.Soff[k]] = -1;
            r += rbar;
        }
        if (tid == 0) *it.rank = r;
    }
}

size_t batched_smem_bytes() { return (size_t)BTAB_WORDS * sizeof(uint64_t); }

cudaError_t launch_batched(cudaStream_t st, const gf2_batch_item *items, const int32_t *order, int count,
                           int32_t *next, uint64_t *scratch, int64_t max_rows, int64_t ldS, int grid)
{
    const size_t per_idx = (size_t)max_rows, per_S = (size_t)SMAX * ldS;
    BatchScratch scr;
    scr.max_rows = max_rows;
    scr.ldS = ldS;
    scr.idx = scratch;
    scr.S = scr.idx + per_idx * grid;
    scr.gval = scr.S + per_S * grid;
    scr.glb = scr.gval + per_idx * grid;
    scr.gsrc = reinterpret_cast<int32_t *>(scr.glb + per_idx * grid);
    batched_ple_kernel<<<grid, BATCH_THREADS, batched_smem_bytes(), st>>>(items, order, count, next, scr);
    return cudaGetLastError();
}

size_t batched_scratch_words(int64_t max_rows, int64_t ldS, int grid)
{
    return ((size_t)max_rows * 3 + (size_t)SMAX * ldS) * grid + ((size_t)max_rows * grid + 1) / 2 + 64;
}

int batched_grid(int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_ple_kernel, BATCH_THREADS,
                                                      batched_smem_bytes()) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    if (per_sm < 1) per_sm = 1;
    return per_sm * num_sms;
}

}  // namespace gf2
