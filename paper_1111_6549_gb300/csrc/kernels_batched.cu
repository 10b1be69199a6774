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
constexpr int BTAB_WORDS = 4096;                     // 32 KiB of tables: the largest configuration
constexpr int BG_WORDS = KS * 4;                     // generator words of a tile: 64 rows x up to 4 words

constexpr int cfg_table_words(int k, int bw) { return (KS / k) * (1 << k) * bw; }
static_assert(cfg_table_words(8, 2) <= BTAB_WORDS && cfg_table_words(8, 1) <= BTAB_WORDS &&
              cfg_table_words(4, 1) <= BTAB_WORDS && cfg_table_words(4, 2) <= BTAB_WORDS &&
              cfg_table_words(4, 4) <= BTAB_WORDS, "table configuration larger than the table buffer");

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

// The tabulated update (Algorithms 5 and 6) of the words [w_lo, W) of every
// row at a position >= r, one tile of BW words at a time: the 64 / K tables of
// a tile hold, for every K-bit value e, the XOR of the generator rows selected
// by e (generators K tau .. K tau + K - 1 for table tau), and each row XORs in
// one entry per table, chosen by the matching K bits of its index word.
template <int K, int BW>
__device__ __forceinline__ void batch_tables_update(uint64_t *T, uint64_t *sG, const uint64_t *S, int64_t ldS,
                                                    uint64_t *A, int64_t ld, int64_t r, int64_t rows, int64_t W,
                                                    int64_t w_lo, int rbar, const int16_t *smap, int maxpos,
                                                    const uint64_t *idx)
{
    constexpr int NT = KS / K, NE = 1 << K;
    const int tid = threadIdx.x;
    for (int64_t wbase = (w_lo / BW) * BW; wbase < W; wbase += BW) {
        for (int t = tid; t < KS * BW; t += BATCH_THREADS) {
            const int g = t / BW, x = t - g * BW;
            sG[t] = (g < rbar && wbase + x < W) ? S[(int64_t)g * ldS + wbase + x] : 0ull;
        }
        __syncthreads();
        for (int e2 = tid; e2 < NT * NE; e2 += BATCH_THREADS) {
            const int tau = e2 >> K, e = e2 & (NE - 1);
            uint64_t acc[BW];
#pragma unroll
            for (int x = 0; x < BW; ++x) acc[x] = 0;
#pragma unroll
            for (int bq = 0; bq < K; ++bq) {
                const uint64_t msk = 0ull - (uint64_t)((e >> bq) & 1);
#pragma unroll
                for (int x = 0; x < BW; ++x) acc[x] ^= sG[(K * tau + bq) * BW + x] & msk;
            }
#pragma unroll
            for (int x = 0; x < BW; ++x) T[(size_t)e2 * BW + x] = acc[x];
        }
        __syncthreads();
        for (int64_t off = tid; off < rows; off += BATCH_THREADS) {
            const int k = (off <= maxpos) ? smap[off] : -1;
            const uint64_t *src = (k >= 0) ? S + (int64_t)k * ldS : A + (r + off) * ld;
            uint64_t *dst = A + (r + off) * ld;
            const uint64_t ix = idx[off];
            uint64_t acc[BW];
#pragma unroll
            for (int x = 0; x < BW; ++x) {
                const int64_t w = wbase + x;
                acc[x] = (w >= w_lo && w < W) ? src[w] : 0ull;
            }
#pragma unroll
            for (int tau = 0; tau < NT; ++tau) {
                const int e = (int)((ix >> (K * tau)) & (uint64_t)(NE - 1));
                const uint64_t *te = T + ((size_t)tau * NE + e) * BW;
                if constexpr (BW % 2 == 0) {
#pragma unroll
                    for (int x = 0; x < BW; x += 2) {
                        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(te + x);
                        acc[x] ^= v.x;
                        acc[x + 1] ^= v.y;
                    }
                } else {
#pragma unroll
                    for (int x = 0; x < BW; ++x) acc[x] ^= te[x];
                }
            }
#pragma unroll
            for (int x = 0; x < BW; ++x) {
                const int64_t w = wbase + x;
                if (w >= w_lo && w < W) dst[w] = acc[x];
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(BATCH_THREADS, 4)
batched_ple_kernel(const gf2_batch_item *items, const int32_t *order, int count, int32_t *next,
                   BatchScratch scr, uint32_t tune_bits)
{
    extern __shared__ __align__(16) uint64_t T[];    // BTAB_WORDS: [table][entry][tile word]
    __shared__ PanelShared sh;
    __shared__ uint64_t sLinv[KS], sMinv[KS], sBx[KS];
    __shared__ int8_t sCol[KS];
    __shared__ int16_t smap[BATCH_MAX_ROWS];          // position offset -> staged slot, or -1
    __shared__ int sh_item;
    __shared__ __align__(16) uint64_t sG[BG_WORDS];   // generator words of the current tile

    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t *idx = scr.idx + (size_t)blockIdx.x * scr.max_rows;
    uint64_t *S = scr.S + (size_t)blockIdx.x * SMAX * scr.ldS;
    PanelScratch gs{scr.gval + (size_t)blockIdx.x * scr.max_rows, scr.glb + (size_t)blockIdx.x * scr.max_rows,
                    scr.gsrc + (size_t)blockIdx.x * 2 * scr.max_rows,
                    scr.gsrc + (size_t)blockIdx.x * 2 * scr.max_rows + scr.max_rows};
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
            // L11^-1 and U11^-1 side by side (the window's register budget
            // here leaves no room to form them during the search)
            if (warp == 0) warp_lower_inverse_blocked(sh.L, rbar, sLinv);
            if (warp == 1) warp_upper_inverse(sh, rbar, T, T + KS, sMinv);   // scratch in T (free here)
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
            // the bases of the row lookups: for a stripe word with bits u on
            // the pivot columns, its L coefficients v = u U11^-1 and its table
            // index v L11^-1 are XORs over the set bits of u of one row per
            // pivot p: row p of U11^-1 and of U11^-1 L11^-1
            if (tid < KS) sCol[tid] = -1;
            __syncthreads();
            if (tid < rbar) {
                const uint64_t mp = sMinv[tid];
                uint64_t x = 0;
                for (int q = 0; q < rbar; ++q) x ^= sLinv[q] & (0ull - ((mp >> q) & 1ull));
                sBx[tid] = x;
                sCol[sh.j[tid]] = (int8_t)tid;
            }
            // the lookup tables in T (free until the update), built level by
            // level: entry e of a byte's table is entry e - 2^l plus the basis
            // row of bit l, for 2^l <= e < 2^(l+1); [kind * 8 + byte][256]
            if (tid < 16) T[tid * 256] = 0ull;
            for (int l = 0; l < 8; ++l) {
                __syncthreads();
                const int cnt = 1 << l;
                for (int e2 = tid; e2 < 16 * cnt; e2 += BATCH_THREADS) {
                    const int tb = e2 >> l, e = cnt + (e2 & (cnt - 1));
                    const int p = sCol[8 * (tb & 7) + l];
                    const uint64_t basis = p < 0 ? 0ull : (tb >= 8 ? sBx[p] : sMinv[p]);
                    T[tb * 256 + e] = T[tb * 256 + e - cnt] ^ basis;
                }
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
                    const uint64_t sw = row[cw];
                    v = 0;
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const int e = (int)((sw >> (8 * b)) & 255ull);
                        v ^= T[b * 256 + e];
                        ix ^= T[(8 + b) * 256 + e];
                    }
                }
                batch_write_lregion(row, r, cw, rbar, v, es);
                idx[off] = ix;
            }
            __syncthreads();
            // tabulated update of the words right of the stripe, in the
            // configuration tuned for this matrix's size class
            switch ((tune_bits >> (4 * batch_size_class(m, n))) & 15u) {
            case 1: batch_tables_update<8, 1>(T, sG, S, ldS, A, ld, r, rows, W, cw + 1, rbar, smap, maxpos, idx); break;
            case 2: batch_tables_update<4, 1>(T, sG, S, ldS, A, ld, r, rows, W, cw + 1, rbar, smap, maxpos, idx); break;
            case 3: batch_tables_update<4, 2>(T, sG, S, ldS, A, ld, r, rows, W, cw + 1, rbar, smap, maxpos, idx); break;
            case 4: batch_tables_update<4, 4>(T, sG, S, ldS, A, ld, r, rows, W, cw + 1, rbar, smap, maxpos, idx); break;
            default: batch_tables_update<8, 2>(T, sG, S, ldS, A, ld, r, rows, W, cw + 1, rbar, smap, maxpos, idx); break;
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

// Random Bernoulli(1/2) contents for tuning batches: splitmix64 of
// (seed, matrix, word), padding bits cleared.
__global__ void batch_fill_kernel(const gf2_batch_item *items, int count, uint64_t seed)
{
    for (int b = blockIdx.x; b < count; b += gridDim.x) {
        const gf2_batch_item it = items[b];
        const int64_t W = (it.n + 63) >> 6;
        const uint64_t pad = (it.n & 63) ? ((1ull << (it.n & 63)) - 1ull) : ~0ull;
        for (int64_t t = threadIdx.x; t < it.m * W; t += blockDim.x) {
            const int64_t i = t / W, w = t - i * W;
            uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(((int64_t)b << 32) + t + 1);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            it.A[i * it.ld_words + w] = (w == W - 1) ? (z & pad) : z;
        }
    }
}

cudaError_t launch_batch_fill(cudaStream_t st, const gf2_batch_item *items, int count, uint64_t seed, int num_sms)
{
    if (count <= 0) return cudaSuccess;
    const int grid = count < 8 * num_sms ? count : 8 * num_sms;
    batch_fill_kernel<<<grid, 256, 0, st>>>(items, count, seed);
    return cudaGetLastError();
}

size_t batched_smem_bytes() { return (size_t)BTAB_WORDS * sizeof(uint64_t); }

cudaError_t launch_batched(cudaStream_t st, const gf2_batch_item *items, const int32_t *order, int count,
                           int32_t *next, uint64_t *scratch, int64_t max_rows, int64_t ldS, int grid,
                           BatchTune tune)
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
    uint32_t tune_bits = 0;                           // 4 bits per size class
    for (int c = 0; c < BATCH_CLASSES; ++c) tune_bits |= (uint32_t)(tune.cfg[c] & 15) << (4 * c);
    // (the dynamic shared-memory limit was raised by batched_grid, which
    // every caller runs first, outside any stream capture)
    batched_ple_kernel<<<grid, BATCH_THREADS, batched_smem_bytes(), st>>>(items, order, count, next, scr,
                                                                          tune_bits);
    return cudaGetLastError();
}

size_t batched_scratch_words(int64_t max_rows, int64_t ldS, int grid)
{
    // per CTA: index, panel values and L bits (8 B per row each), staged rows,
    // panel sources and positions (2 x 4 B per row)
    return ((size_t)max_rows * 4 + (size_t)SMAX * ldS) * grid + 64;
}

int batched_grid(int num_sms)
{
    int per_sm = 0;
    if (cudaFuncSetAttribute(batched_ple_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batched_smem_bytes()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_ple_kernel, BATCH_THREADS,
                                                      batched_smem_bytes()) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    if (per_sm < 1) per_sm = 1;
    return per_sm * num_sms;
}

}  // namespace gf2
