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
#include "panel_dev.cuh"

namespace gf2 {

__global__ void init_ple_kernel(int64_t *P, int64_t *Q, int64_t m, int64_t qn, int32_t *map,
                                int64_t *r_dev)
{
    pdl_wait();
    pdl_trigger();
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
    return launch_kernel(init_ple_kernel, dim3((int)blocks), dim3(256), 0, st, P, Q, m, qn, map, r_dev);
}

__global__ void __launch_bounds__(PANEL_THREADS)
panel_kernel(const uint64_t *__restrict__ A, int64_t m, int64_t ld, int64_t npiv, int s,
             StripeDesc *descs, int64_t *r_dev, int64_t *P, int64_t *Q, int32_t *map,
             PanelScratch gs, int32_t *fallbacks, uint64_t *ptab, const int32_t *prev_map,
             const uint64_t *prev_S, int64_t ldS)
{
    pdl_wait();
    pdl_trigger();
    __shared__ PanelShared sh;
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
    // with the previous stripe's update still running, the rows its swaps
    // moved are read from its staged copies
    PrevStage ps{nullptr, prev_S, ldS, 0, -1, s - 1};
    if (prev_map && s > 0) {
        const StripeDesc *dp = descs + (s - 1);
        if (dp->rbar > 0) {
            ps.map = prev_map;
            ps.r = dp->r;
            ps.maxpos = dp->maxpos;
        }
    }
    if (warp < 4) panel_window4(A, r, ld, cw, rows, keff, sh, ps);
    __syncthreads();
    const bool fell_back = sh.fail != 0;
    if (fell_back) panel_block(A, r, ld, cw, rows, keff, gs, sh, fallbacks, ps);

    // ---------------- outputs
    const int rbar = sh.rbar;
    __shared__ uint64_t sMinv[KS], sLinv[KS];          // shared copies for the prep tables
    if (warp == 1) {
        // U11^-1 for the RREF recovery, beside warp 0's L11^-1
        __shared__ uint64_t sU[KS], sUi[KS];
        warp_upper_inverse(sh, rbar, sU, sUi, sMinv);
        __syncwarp();
        for (int p = lane; p < rbar; p += 32) d->Minv[p] = sMinv[p];
    }
    if (warp == 0) warp_lower_inverse_blocked(sh.L, rbar, d->Linv, sLinv);
    for (int p = tid; p < rbar; p += blockDim.x) {
        P[r + p] = r + sh.t[p];
        Q[r + p] = c + sh.j[p];
        d->E11[p] = sh.E[p];
        d->L11[p] = sh.L[p];
        d->qbar[p] = sh.j[p];
    }
    const int nS = sh.nS;
    for (int k = tid; k < nS; k += blockDim.x) {
        d->S_off[k] = sh.Soff[k];
        d->S_src[k] = sh.Ssrc[k];
        map[r + sh.Soff[k]] = s * 256 + k;
    }
    if (tid == 0) {
        d->r = r; d->rbar = rbar; d->c = c; d->nS = nS; d->maxpos = sh.maxpos;
        d->tier = sh.fail ? 2 : 1;
        *r_dev = r + rbar;
    }
    if (ptab == nullptr) return;
    // The bases of the prep kernel's tables: for a stripe word with bits u on
    // the pivot columns, the L coefficients v = u U11^-1, the table index
    // v L11^-1 and the word rebuilt from the pivot bits (u U11^-1 E11) are
    // XORs over the word's set bits of one basis row per stripe column: row
    // p of U11^-1, of U11^-1 L11^-1 and of U11^-1 E11 for the column's pivot
    // p (zero for a column without one).
    static_assert(PANEL_THREADS == 8 * KS, "eight threads per pivot for the bases");
    __shared__ uint64_t tB[3][KS];
    if (tid < KS) {
        tB[0][tid] = 0ull;
        tB[1][tid] = 0ull;
        tB[2][tid] = 0ull;
    }
    __syncthreads();                                   // Minv and Linv are written
    {
        // pivot p's two sums over U11^-1's row, eight threads (one warp
        // quarter) per pivot, eight terms each, folded by shuffles
        const int p = tid >> 3, part = tid & 7;
        const uint64_t mp = p < rbar ? sMinv[p] : 0ull;
        uint64_t x = 0, g = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int q = 8 * part + i;
            const uint64_t sel = (q < rbar) ? 0ull - ((mp >> q) & 1ull) : 0ull;
            x ^= sLinv[q] & sel;
            g ^= sh.E[q] & sel;
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            x ^= __shfl_xor_sync(0xffffffffu, x, o);
            g ^= __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (part == 0 && p < rbar) {
            const int col = sh.j[p];
            tB[0][col] = mp;
            tB[1][col] = x;
            tB[2][col] = g;
        }
    }
    __syncthreads();
    if (tid < 3 * KS) ptab[tid] = tB[tid / KS][tid % KS];   // [kind][column]: the prep builds its tables from them
}

cudaError_t launch_panel(cudaStream_t st, uint64_t *A, int64_t m, int64_t ld, int64_t npiv, int s,
                         StripeDesc *descs, int64_t *r_dev, int64_t *P, int64_t *Q, int32_t *map,
                         PanelScratch gs, int32_t *fallbacks, uint64_t *ptab, const int32_t *prev_map,
                         const uint64_t *prev_S, int64_t ldS)
{
    return launch_kernel(panel_kernel, dim3(1), dim3(PANEL_THREADS), 0, st, (const uint64_t *)A, m, ld, npiv, s, descs,
                         r_dev, P, Q, map, gs, fallbacks, ptab, prev_map, prev_S, ldS);
}

// ----------------------------------------------------------------------------
// prep

// The L region of one row (columns r .. r+rbar-1 get the L bits v, word cw
// the stripe word es), from values already loaded: wkeep is the row's word
// r/64, whose bits below column r are kept.  Words strictly between the L
// bits and the stripe are zero already and stay zero.
__device__ __forceinline__ void store_lregion(uint64_t *row, int64_t r, int64_t cw, int rbar, uint64_t v,
                                              uint64_t es, uint64_t wkeep)
{
    const int64_t wr = r >> 6;
    const int64_t wl = (r + rbar - 1) >> 6;
    for (int64_t w = wr; w <= wl; ++w) {
        const int64_t off = r - (w << 6);
        uint64_t part = (off >= 0) ? (v << off) : (v >> (-off));
        const uint64_t keep = (w == wr) ? (wkeep & ((1ull << (r & 63)) - 1ull)) : 0ull;
        if (w == cw) part |= es;
        row[w] = keep | part;
    }
    if (cw > wl) row[cw] = es;
}

// XOR over the warp's lanes (every lane gets the total).
__device__ __forceinline__ uint64_t warp_xor(uint64_t x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x ^= __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

constexpr int PREP_THREADS = 512;
constexpr int PREP_STAGE_BLOCKS = SMAX;   // one block per staged row
constexpr int PREP_FIRST_ROW_BLOCK = PREP_STAGE_BLOCKS;
constexpr int PREP_NTAB = 32;             // 3 kinds x 8 bytes of the stripe word, 8 bytes of the index
constexpr size_t PREP_SMEM = (size_t)PREP_NTAB * 256 * sizeof(uint64_t);
static_assert(PREP_THREADS == 16 * 32, "one warp per two tables");

__global__ void __launch_bounds__(PREP_THREADS)
prep_kernel(uint64_t *A, int64_t m, int64_t ld, int64_t W, int s, StripeDesc *descs,
            const int32_t *map, uint64_t *S, int64_t ldS, uint64_t *IDX, int32_t *err,
            const uint64_t *__restrict__ ptab, int64_t nw)
{
    pdl_wait();
    pdl_trigger();
    const StripeDesc *d = descs + s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the bases by stripe column (kind 0: L coefficients, 1: table index, 2:
    // rebuilt word) and word nw of the raw pivot rows by pivot index (their
    // sources, which no CTA writes here); the loads that do not depend on the
    // stripe record go out beside it
    __shared__ uint64_t sB[3][KS], sG[KS];
    uint64_t b0 = 0, b1 = 0, b2 = 0;
    int64_t src = 0;
    if (tid < KS) {
        b0 = ptab[tid];
        b1 = ptab[KS + tid];
        b2 = ptab[2 * KS + tid];
        src = d->S_src[tid];
    }
    const int rbar = d->rbar;
    if (rbar == 0) return;
    const int64_t r = d->r;
    const int64_t cw = d->c >> 6;
    const int nS = d->nS;
    const int maxpos = d->maxpos;
    const int64_t wr = r >> 6;                       // the word holding column r
    // a row CTA's first row per thread: its words (the stripe word, the next
    // word, the word holding column r) and its map entry load beside the
    // pivot rows' words below
    const bool rowblk = blockIdx.x >= PREP_STAGE_BLOCKS;
    const int64_t i0 = r + (int64_t)(blockIdx.x - PREP_FIRST_ROW_BLOCK) * blockDim.x + tid;
    uint64_t sw0 = 0, wn0 = 0, wk0 = 0;
    int mv0 = -1;
    if (rowblk && i0 < m) {
        const uint64_t *row = A + i0 * ld;
        sw0 = row[cw];
        wn0 = nw >= 0 ? row[nw] : 0ull;
        wk0 = wr == cw ? 0ull : row[wr];
        if (i0 - r <= maxpos) mv0 = map[i0];
    }
    if (tid < KS) {
        sB[0][tid] = b0;
        sB[1][tid] = b1;
        sB[2][tid] = b2;
        sG[tid] = (tid < rbar && nw >= 0) ? A[src * ld + nw] : 0ull;
    }
    __syncthreads();

    if (blockIdx.x < PREP_STAGE_BLOCKS) {
        // staged rows: copy the whole source row (keeping the words the
        // lookups need), then fix its L region
        __shared__ uint64_t sw3[3];                  // words cw, nw and r / 64 of the row
        for (int k = blockIdx.x; k < nS; k += PREP_STAGE_BLOCKS) {   // at most one per block
            const uint64_t *__restrict__ srow = A + d->S_src[k] * ld;
            uint64_t *__restrict__ dst = S + (int64_t)k * ldS;
            // four words per thread loaded before any is stored (one round
            // trip up to 2048 words)
            for (int64_t wb = tid; wb < W; wb += 4 * (int64_t)blockDim.x) {
                uint64_t x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t w = wb + (int64_t)u * blockDim.x;
                    x[u] = w < W ? srow[w] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t w = wb + (int64_t)u * blockDim.x;
                    if (w >= W) break;
                    dst[w] = x[u];
                    if (w == cw) sw3[0] = x[u];
                    if (w == nw) sw3[1] = x[u];
                    if (w == wr) sw3[2] = x[u];
                }
            }
            __syncthreads();
            if (warp == 0) {
                const int64_t pos = r + d->S_off[k];
                const uint64_t sw = sw3[0];
                uint64_t v, es, ix;
                if (k < rbar) {
                    v = d->L11[k];
                    es = d->E11[k];
                    ix = d->Linv[k] ^ (1ull << k);
                } else {
                    // a displaced row: the bases of its set bits, summed over the warp
                    uint64_t g = 0;
                    v = 0;
                    ix = 0;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int col = lane + 32 * h;
                        if ((sw >> col) & 1ull) {
                            v ^= sB[0][col];
                            ix ^= sB[1][col];
                            g ^= sB[2][col];
                        }
                    }
                    v = warp_xor(v);
                    ix = warp_xor(ix);
                    g = warp_xor(g);
                    if (lane == 0 && g != sw && err) atomicExch(err, 1);
                    es = 0;
                }
                // the stripe's update of word nw: the raw pivot rows selected by ix
                uint64_t nx = 0;
                if (nw >= 0) {
                    nx = (((ix >> lane) & 1ull) ? sG[lane] : 0ull) ^ (((ix >> (lane + 32)) & 1ull) ? sG[lane + 32] : 0ull);
                    nx = warp_xor(nx);
                }
                if (lane == 0) {
                    store_lregion(dst, r, cw, rbar, v, es, sw3[2]);
                    if (nw >= 0) dst[nw] = sw3[1] ^ nx;
                    IDX[pos] = ix;
                }
            }
            __syncthreads();
        }
        return;
    }
    // Every other row at a position >= r: its L coefficients, its table
    // index and its stripe word rebuilt from its pivot-column bits, each as
    // eight lookups by the bytes of the stripe word, and the update of word
    // nw as eight lookups by the bytes of the index.  The 32 tables are
    // built here in shared memory, warp w forming tables 2w and 2w+1: entry
    // 32 h + lane is the XOR of the basis rows of the low five bits (lane)
    // and of the high three (h), so every store covers 32 consecutive words
    // (no bank conflicts).  A row whose word is not rebuilt exactly lies
    // outside the span of E11: an internal error.
    extern __shared__ __align__(16) uint64_t T[];           // [kind * 8 + byte][256]
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int tb = 2 * warp + half, kind = tb >> 3, c0 = 8 * (tb & 7);
        const uint64_t *base = kind < 3 ? sB[kind] + c0 : sG + c0;   // index byte: raw pivot rows c0 ..
        uint64_t lo = 0;
#pragma unroll
        for (int l = 0; l < 5; ++l) lo ^= ((lane >> l) & 1) ? base[l] : 0ull;
        uint64_t hv[8];
        hv[0] = 0ull;
        hv[1] = base[5];
        hv[2] = base[6];
        hv[3] = base[5] ^ base[6];
#pragma unroll
        for (int h = 0; h < 4; ++h) hv[4 + h] = hv[h] ^ base[7];
#pragma unroll
        for (int h = 0; h < 8; ++h) T[tb * 256 + 32 * h + lane] = hv[h] ^ lo;
    }
    __syncthreads();
    const int64_t stride = (int64_t)(gridDim.x - PREP_FIRST_ROW_BLOCK) * blockDim.x;
    for (int64_t i = i0; i < m; i += stride) {
        // the row's words in one round trip (the first row's already loaded):
        // the stripe word, the next word, and the word holding column r (the
        // stripe word itself at full rank)
        uint64_t sw, wn, wk;
        int mv;
        uint64_t *row = A + i * ld;
        if (i == i0) {
            sw = sw0;
            wn = wn0;
            wk = wk0;
            mv = mv0;
        } else {
            sw = row[cw];
            wn = nw >= 0 ? row[nw] : 0ull;
            wk = wr == cw ? 0ull : row[wr];
            mv = i - r <= maxpos ? map[i] : -1;
        }
        if (wr == cw) wk = sw;
        if (mv >= 0 && (mv >> 8) == s) continue;           // staged row
        uint64_t v = 0, ix = 0, g = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int e = (int)((sw >> (8 * b)) & 255ull);
            v ^= T[b * 256 + e];
            ix ^= T[(8 + b) * 256 + e];
            g ^= T[(16 + b) * 256 + e];
        }
        if (g != sw && err) atomicExch(err, 1);
        store_lregion(row, r, cw, rbar, v, 0ull, wk);
        if (nw >= 0) {
            uint64_t nx = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) nx ^= T[(24 + b) * 256 + (int)((ix >> (8 * b)) & 255ull)];
            row[nw] = wn ^ nx;
        }
        IDX[i] = ix;
    }
}

cudaError_t setup_prep_kernel()
{
    return cudaFuncSetAttribute(prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PREP_SMEM);
}

cudaError_t launch_prep(cudaStream_t st, uint64_t *A, int64_t m, int64_t ld, int64_t W, int s,
                        StripeDesc *descs, const int32_t *map, uint64_t *S, int64_t ldS,
                        uint64_t *IDX, int32_t *err, const uint64_t *ptab, int num_sms, int64_t next_word)
{
    // row blocks: at most one per SM (each builds its own 64 KiB of tables)
    int64_t blocks = (m + PREP_THREADS - 1) / PREP_THREADS;
    if (blocks < 1) blocks = 1;
    if (blocks > num_sms) blocks = num_sms;
    return launch_kernel(prep_kernel, dim3((int)(blocks + PREP_FIRST_ROW_BLOCK)), dim3(PREP_THREADS), PREP_SMEM, st, A, m, ld,
                         W, s, descs, map, S, ldS, IDX, err, ptab, next_word);
}

}  // namespace gf2
