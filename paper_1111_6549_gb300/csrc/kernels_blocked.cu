// kernels_blocked.cu -- helpers of the blocked PLE, where the trailing update
// of a block of stripes is one large GF(2) product instead of one table pass
// per stripe (the structure of Algorithm 3's A11 += A10 A01 step, iterated
// over column blocks).
//
// After the stripes of a column block [c0, c1) have been decomposed with
// their updates restricted to the block, the rows [r0, r1) hold the block's
// pivots and every row's L bits for these pivots sit in the bit columns
// [r0, r1).  The columns right of the block then need
//     U = L11^-1 A[r0:r1, right]               (TRSM, pivot rows)
//     A[r1:m, right] ^= L21 U                   (product, rows below)
// gather_lbits_kernel copies the L bits [r0, r1) of rows r0.. into an aligned
// buffer (the GEMM and TRSM operands); the TRSM halves recursively through
// gf2_mul down to leaves of at most 4096 rows, each solved by one fused launch
// (trsm_leaf_kernel).
#include "panel_dev.cuh"

#include <algorithm>
#include <climits>

namespace gf2 {

// out[i][w] = bits [c0 + 64 w, c0 + 64 w + 64) of row row0 + i, masked to the
// first kb bits (i < rows, w < kw)
__global__ void gather_lbits_kernel(const uint64_t *__restrict__ A, int64_t ld, int64_t W, int64_t row0,
                                    int64_t rows, int64_t c0, int64_t kb, int64_t kw, uint64_t *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const int64_t total = rows * kw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / kw, w = t - i * kw;
        const uint64_t *row = A + (row0 + i) * ld;
        const int64_t b = c0 + 64 * w;                  // first bit
        const int64_t q = b >> 6;
        const int off = (int)(b & 63);
        uint64_t v = row[q] >> off;
        if (off && q + 1 < W) v |= row[q + 1] << (64 - off);
        const int64_t left = kb - 64 * w;               // bits of this word that belong to the block
        if (left < 64) v &= (1ull << left) - 1ull;
        out[i * kw + w] = v;
    }
}

cudaError_t launch_gather_lbits(cudaStream_t st, const uint64_t *A, int64_t ld, int64_t W, int64_t row0, int64_t rows,
                                int64_t c0, int64_t kb, int64_t kw, uint64_t *out, int num_sms)
{
    int64_t blocks = (rows * kw + 255) / 256;
    if (blocks > 8 * num_sms) blocks = 8 * num_sms;
    if (blocks < 1) blocks = 1;
    return launch_kernel(gather_lbits_kernel, dim3((int)blocks), dim3(256), 0, st, A, ld, W, row0, rows, c0, kb, kw,
                         out);
}

// out[i][w] = the bits of row row0 + i at the columns Qb[64 w .. 64 w + 64)
// (bit b of word w from column Qb[64 w + b]) for the first kb entries of the
// increasing column list Qb (i < rows, w < kw).  A word whose 64 columns are
// consecutive is one shifted load; the others go bit by bit.
__global__ void gather_pivbits_kernel(const uint64_t *__restrict__ A, int64_t ld, int64_t W, int64_t row0,
                                      int64_t rows, const int64_t *__restrict__ Qb, int64_t kb, int64_t kw,
                                      uint64_t *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const int64_t total = rows * kw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / kw, w = t - i * kw;
        const uint64_t *row = A + (row0 + i) * ld;
        const int64_t nb = kb - 64 * w < 64 ? kb - 64 * w : 64;
        const int64_t qf = __ldg(Qb + 64 * w), ql = __ldg(Qb + 64 * w + nb - 1);
        uint64_t v = 0;
        if (ql - qf == nb - 1) {
            const int64_t q = qf >> 6;
            const int off = (int)(qf & 63);
            v = row[q] >> off;
            if (off && q + 1 < W) v |= row[q + 1] << (64 - off);
            if (nb < 64) v &= (1ull << nb) - 1ull;
        } else {
            for (int b = 0; b < nb; ++b) {
                const int64_t c = __ldg(Qb + 64 * w + b);
                v |= ((row[c >> 6] >> (c & 63)) & 1ull) << b;
            }
        }
        out[i * kw + w] = v;
    }
}

cudaError_t launch_gather_pivbits(cudaStream_t st, const uint64_t *A, int64_t ld, int64_t W, int64_t row0,
                                  int64_t rows, const int64_t *Qb, int64_t kb, int64_t kw, uint64_t *out,
                                  int num_sms)
{
    int64_t blocks = (rows * kw + 255) / 256;
    if (blocks > 8 * num_sms) blocks = 8 * num_sms;
    if (blocks < 1) blocks = 1;
    return launch_kernel(gather_pivbits_kernel, dim3((int)blocks), dim3(256), 0, st, A, ld, W, row0, rows, Qb, kb, kw,
                         out);
}

// ---------------------------------------------------------------------------
// Fused TRSM leaf: X <- L^-1 X for the kb <= TRSM_LEAF_MAX rows X = A[row0 ..
// row0 + kb) over the words [w_lo, W), L unit lower triangular with its
// strictly lower bits gathered in Lt (kb x ldt words).  Forward substitution
// in steps of 64 rows: step t replaces rows 64 t .. 64 t + 63 by their
// product with the inverse of L's diagonal block t and adds to every row
// below its L bits in block t times those new rows.  Both are one table
// lookup per row on tables built from the step's rows as they stand before
// the step (the index of a diagonal row p is row p of the block inverse
// plus e_p; of a row below, its L bits times the block inverse), so a whole
// leaf is one launch: columns are independent, each CTA owns two words of
// every row and walks all steps alone.  trsm_leaf_prep_kernel forms the
// indices, one CTA per step.

constexpr int LEAF_THREADS = 256;

// Lp[t * kb + i] for the rows i >= 64 t of the leaf: the index of row i in
// step t (as above).
__global__ void __launch_bounds__(LEAF_THREADS)
trsm_leaf_prep_kernel(const uint64_t *__restrict__ Lt, int64_t ldt, int64_t kb, uint64_t *__restrict__ Lp)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint64_t sL[KS], sM[KS];
    __shared__ uint64_t tab[8][256];
    const int t = blockIdx.x, tid = threadIdx.x;
    const int nt = (int)min((int64_t)KS, kb - 64 * (int64_t)t);
    if (tid < KS) sL[tid] = (tid < nt) ? (Lt[(64 * (int64_t)t + tid) * ldt + t] & ((1ull << tid) - 1ull)) : 0ull;
    __syncthreads();
    if (tid < 32) warp_lower_inverse_blocked(sL, nt, sM);
    __syncthreads();
    // byte tables of the block inverse's rows: tab[b][e] = XOR of rows 8 b + q, bits q of e
    for (int e2 = tid; e2 < 8 * 256; e2 += blockDim.x) {
        const int b = e2 >> 8, e = e2 & 255;
        uint64_t acc = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (((e >> q) & 1) && 8 * b + q < nt) acc ^= sM[8 * b + q];
        tab[b][e] = acc;
    }
    __syncthreads();
    const uint64_t vmask = nt == 64 ? ~0ull : ((1ull << nt) - 1ull);
    for (int64_t i = 64 * (int64_t)t + tid; i < kb; i += blockDim.x) {
        const int64_t off = i - 64 * (int64_t)t;
        uint64_t v;
        if (off < nt) {
            v = sM[off] ^ (1ull << off);
        } else {
            const uint64_t x = Lt[i * ldt + t] & vmask;
            v = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) v ^= tab[b][(x >> (8 * b)) & 255u];
        }
        Lp[(int64_t)t * kb + i] = v;
    }
}

// One CTA per pair of words; see the comment above.  The CTA's two words of
// the leaf's rows (at most TRSM_LEAF_MAX x 16 bytes) stay in shared memory
// for all steps: loaded once, updated in place, stored once.  Thread t owns
// the rows t, t + 256, ... in every step, so it loads the next step's
// indices of its rows while the current step runs.
//
// Shared-memory banks.  A 16-byte access of a warp is served in four phases
// of eight lanes; a phase costs one wavefront when its eight lanes fall into
// eight different groups of four banks.  The tables are laid out entry-major,
// T[8 e + t] for entry e of table t, so the slot of table t is always in bank
// group t.  A row's eight lookups are taken in an order rotated by its lane
// (round k reads table (k + lane) mod 8), so the eight lanes of a phase read
// eight different tables whatever their indices are.  The build keeps the
// same property: lane l writes table l mod 8, entries 32 w + 4 g + l / 8 of
// warp w in Gray-code order g, from the step's rows kept at slot 9 t + b for
// row 8 t + b (bank group t + b, distinct across the eight tables of a
// phase).
constexpr int LEAF_RPT_MAX = (int)(TRSM_LEAF_MAX / LEAF_THREADS);
static_assert(LEAF_THREADS == 256, "the table build gives each of eight warps 32 entries of every table");

__device__ __forceinline__ uint64_t rotr64(uint64_t x, int s)
{
    return s == 0 ? x : (x >> s) | (x << (64 - s));
}

template <int RPT>
__global__ void __launch_bounds__(LEAF_THREADS)
trsm_leaf_kernel(uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *__restrict__ Lp, int64_t w_lo,
                 int64_t W)
{
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) ulonglong2 T[256 * 8];         // eight 8-bit tables, entry-major
    __shared__ __align__(16) ulonglong2 Gp[72];             // the step's rows: row 8 t + b at slot 9 t + b
    extern __shared__ __align__(16) ulonglong2 Xs[];        // [row]: the CTA's two words of the leaf's rows
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t w0 = w_lo + 2 * (int64_t)blockIdx.x;
    if (w0 >= W) return;
    const bool two = w0 + 1 < W;
    uint64_t *X = A + row0 * ld + w0;
    for (int u = 0; u < RPT; ++u) {
        const int64_t i = tid + (int64_t)u * LEAF_THREADS;
        if (i < kb) Xs[i] = make_ulonglong2(X[i * ld], two ? X[i * ld + 1] : 0ull);
    }
    const int nsteps = (int)((kb + 63) / 64);
    const int rot = 8 * (lane & 7);
    uint64_t ixn[RPT];                                      // the indices of this thread's rows, one step ahead
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int64_t i = tid + (int64_t)u * LEAF_THREADS;
        ixn[u] = (i < kb) ? __ldg(Lp + i) : 0ull;
    }
    for (int t = 0; t < nsteps; ++t) {
        const int64_t r0 = 64 * (int64_t)t;
        const int nt = (int)min((int64_t)KS, kb - r0);
        __syncthreads();                                    // rows of this step written by the last one
        if (tid < KS) {
            const ulonglong2 z = make_ulonglong2(0ull, 0ull);
            Gp[9 * (tid >> 3) + (tid & 7)] = tid < nt ? Xs[r0 + tid] : z;
        }
        uint64_t ix[RPT];
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            ix[u] = ixn[u];
            const int64_t i = tid + (int64_t)u * LEAF_THREADS;
            ixn[u] = (t + 1 < nsteps && i >= r0 + 64 && i < kb) ? __ldg(Lp + (int64_t)(t + 1) * kb + i) : 0ull;
        }
        __syncthreads();
        {
            const int tt = lane & 7, sub = lane >> 3;
            const ulonglong2 *g = Gp + 9 * tt;
            uint64_t v0 = 0, v1 = 0;
            auto add = [&](int c) {
                const ulonglong2 x = g[c];
                v0 ^= x.x;
                v1 ^= x.y;
            };
            if (sub & 1) add(0);
            if (sub & 2) add(1);
            if (warp & 1) add(5);
            if (warp & 2) add(6);
            if (warp & 4) add(7);
            int e = 32 * warp + sub;
            T[8 * e + tt] = make_ulonglong2(v0, v1);
#pragma unroll
            for (int j = 1; j < 8; ++j) {
                // Gray code: step j flips bit b = number of trailing zeros of j (entry bit 2 + b)
                const int b = (j & 1) ? 0 : (j & 2) ? 1 : 2;
                add(2 + b);
                e ^= 4 << b;
                T[8 * e + tt] = make_ulonglong2(v0, v1);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int64_t i = tid + (int64_t)u * LEAF_THREADS;
            if (i < r0 || i >= kb) continue;
            ulonglong2 x = Xs[i];
            const uint64_t ir = rotr64(ix[u], rot);         // byte k: the index byte of table (k + lane) mod 8
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = (int)((ir >> (8 * k)) & 255u);
                const ulonglong2 tv = T[8 * e + ((k + lane) & 7)];
                x.x ^= tv.x;
                x.y ^= tv.y;
            }
            Xs[i] = x;
        }
    }
    __syncthreads();
    for (int u = 0; u < RPT; ++u) {
        const int64_t i = tid + (int64_t)u * LEAF_THREADS;
        if (i < kb) {
            const ulonglong2 x = Xs[i];
            X[i * ld] = x.x;
            if (two) X[i * ld + 1] = x.y;
        }
    }
}

cudaError_t launch_trsm_leaf(cudaStream_t st, uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *Lt,
                             int64_t ldt, uint64_t *Lp, int64_t w_lo, int64_t W)
{
    if (kb <= 0 || kb > TRSM_LEAF_MAX || w_lo >= W) return cudaSuccess;
    cudaError_t e =
        launch_kernel(trsm_leaf_prep_kernel, dim3((int)((kb + 63) / 64)), dim3(LEAF_THREADS), 0, st, Lt, ldt, kb, Lp);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((W - w_lo + 1) / 2));
    const size_t smem = (size_t)kb * sizeof(ulonglong2);
    const uint64_t *Lpc = Lp;
    if (kb <= 4 * LEAF_THREADS)
        return launch_kernel(trsm_leaf_kernel<4>, grid, dim3(LEAF_THREADS), smem, st, A, ld, row0, kb, Lpc, w_lo, W);
    if (kb <= 8 * LEAF_THREADS)
        return launch_kernel(trsm_leaf_kernel<8>, grid, dim3(LEAF_THREADS), smem, st, A, ld, row0, kb, Lpc, w_lo, W);
    return launch_kernel(trsm_leaf_kernel<LEAF_RPT_MAX>, grid, dim3(LEAF_THREADS), smem, st, A, ld, row0, kb, Lpc,
                         w_lo, W);
}

// ---------------------------------------------------------------------------
// Fused RREF leaf: the back-substitution of one base block of the RREF
// recovery in one launch.  The block's pivot rows X = A[row0 .. row0 + kb)
// are in echelon form; T, their bits on their own pivot columns, is unit
// upper triangular, and the reduced rows are T^-1 X (they then hold the
// identity on those columns and span the same rows).  Backward substitution
// in steps of 64 rows from the last: step j replaces rows 64 j .. 64 j + 63
// by their product with the inverse of T's diagonal block j and adds to every
// row above its bits on that block's pivot columns times those new rows.  A
// row's bits on the pivot columns of a later step are never changed by the
// steps after it (the rows added are zero left of their own pivots), so
// every step's table index is known from the unreduced block:
// rref_leaf_prep_kernel forms them all from the gathered bits (one CTA per
// step), and rref_leaf_kernel walks the steps with each CTA owning two words
// of every row, as the TRSM leaf does.  A step whose first pivot column lies
// right of a CTA's words changes nothing there, so a CTA starts at the last
// step that reaches its words.

// Lp[j * kb + i] for the rows i < 64 j + 64 of the block: the index of row i
// in step j.  Xb holds the gathered bits (row i, bit q of word w: row i's bit
// on pivot column 64 w + q of the block), kw words per row.
__global__ void __launch_bounds__(LEAF_THREADS)
rref_leaf_prep_kernel(const uint64_t *__restrict__ Xb, int64_t kw, int64_t kb, uint64_t *__restrict__ Lp)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint64_t sR[KS], sM[KS], sUi[KS];
    __shared__ uint64_t tab[8][256];
    const int j = blockIdx.x, tid = threadIdx.x;
    const int64_t r0 = 64 * (int64_t)j;
    const int nt = (int)min((int64_t)KS, kb - r0);
    // the diagonal block reversed (row and column order), a unit lower
    // triangular matrix R with R^-1 the reversal of the block's inverse;
    // rows past the block's end are identity rows
    if (tid < KS) {
        const int p = KS - 1 - tid;
        const uint64_t u = p < nt ? Xb[(r0 + p) * kw + j] : (1ull << p);
        sR[tid] = __brevll(u);
    }
    __syncthreads();
    if (tid < 32) warp_lower_inverse_blocked(sR, KS, sM);
    __syncthreads();
    if (tid < KS) sUi[tid] = __brevll(sM[KS - 1 - tid]);
    __syncthreads();
    for (int e2 = tid; e2 < 8 * 256; e2 += blockDim.x) {
        const int b = e2 >> 8, e = e2 & 255;
        uint64_t acc = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (((e >> q) & 1) && 8 * b + q < nt) acc ^= sUi[8 * b + q];
        tab[b][e] = acc;
    }
    __syncthreads();
    const uint64_t vmask = nt == 64 ? ~0ull : ((1ull << nt) - 1ull);
    for (int64_t i = tid; i < r0 + nt; i += blockDim.x) {
        uint64_t v;
        if (i >= r0) {
            const int off = (int)(i - r0);
            v = sUi[off] ^ (1ull << off);
        } else {
            const uint64_t x = Xb[i * kw + j] & vmask;
            v = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) v ^= tab[b][(x >> (8 * b)) & 255u];
        }
        Lp[(int64_t)j * kb + i] = v;
    }
}

constexpr int RLEAF_THREADS = 512;
constexpr int RLEAF_RPT = (int)(RREF_LEAF_MAX / RLEAF_THREADS);

// One CTA per pair of words [w0, w0 + 2) of [w_lo, w_hi); Qb: the block's
// pivot columns (increasing), or null when the words are not the matrix's
// own (a compacted column set: every step reaches every word).  Layout of the
// tables and of the step's rows as in trsm_leaf_kernel (conflict-free lookups
// and build).
__global__ void __launch_bounds__(RLEAF_THREADS, 1)
rref_leaf_kernel(uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *__restrict__ Lp,
                 const int64_t *__restrict__ Qb, int64_t w_lo, int64_t w_hi)
{
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) ulonglong2 T[256 * 8];
    __shared__ __align__(16) ulonglong2 Gp[72];
    extern __shared__ __align__(16) ulonglong2 Xs[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t w0 = w_lo + 2 * (int64_t)blockIdx.x;
    if (w0 >= w_hi) return;
    const bool two = w0 + 1 < w_hi;
    const int64_t wlast = two ? w0 + 1 : w0;
    // the last step whose rows reach these words (their first pivot column
    // at or before the last word)
    const int nsteps = (int)((kb + 63) / 64);
    int jmax = Qb ? -1 : nsteps - 1;
    if (Qb) {
        int lo = 0, hi = nsteps - 1;                     // largest j with Qb[64 j] / 64 <= wlast
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            if ((__ldg(Qb + 64 * (int64_t)mid) >> 6) <= wlast) { jmax = mid; lo = mid + 1; }
            else hi = mid - 1;
        }
    }
    if (jmax < 0) return;
    const int64_t nrow = min(kb, 64 * (int64_t)jmax + 64);   // rows that steps 0 .. jmax touch
    uint64_t *X = A + row0 * ld + w0;
#pragma unroll
    for (int u = 0; u < RLEAF_RPT; ++u) {
        const int64_t i = tid + (int64_t)u * RLEAF_THREADS;
        if (i < nrow) Xs[i] = make_ulonglong2(X[i * ld], two ? X[i * ld + 1] : 0ull);
    }
    const int rot = 8 * (lane & 7);
    uint64_t ixn[RLEAF_RPT];
#pragma unroll
    for (int u = 0; u < RLEAF_RPT; ++u) {
        const int64_t i = tid + (int64_t)u * RLEAF_THREADS;
        ixn[u] = (i < nrow) ? __ldg(Lp + (int64_t)jmax * kb + i) : 0ull;
    }
    for (int j = jmax; j >= 0; --j) {
        const int64_t r0 = 64 * (int64_t)j;
        const int nt = (int)min((int64_t)KS, kb - r0);
        __syncthreads();                                 // rows of this step written by the last one
        if (tid < KS) {
            const ulonglong2 z = make_ulonglong2(0ull, 0ull);
            Gp[9 * (tid >> 3) + (tid & 7)] = tid < nt ? Xs[r0 + tid] : z;
        }
        uint64_t ix[RLEAF_RPT];
#pragma unroll
        for (int u = 0; u < RLEAF_RPT; ++u) {
            ix[u] = ixn[u];
            const int64_t i = tid + (int64_t)u * RLEAF_THREADS;
            ixn[u] = (j > 0 && i < r0) ? __ldg(Lp + (int64_t)(j - 1) * kb + i) : 0ull;
        }
        __syncthreads();
        if (warp < 8) {
            const int tt = lane & 7, sub = lane >> 3;
            const ulonglong2 *g = Gp + 9 * tt;
            uint64_t v0 = 0, v1 = 0;
            auto add = [&](int c) {
                const ulonglong2 x = g[c];
                v0 ^= x.x;
                v1 ^= x.y;
            };
            if (sub & 1) add(0);
            if (sub & 2) add(1);
            if (warp & 1) add(5);
            if (warp & 2) add(6);
            if (warp & 4) add(7);
            int e = 32 * warp + sub;
            T[8 * e + tt] = make_ulonglong2(v0, v1);
#pragma unroll
            for (int s = 1; s < 8; ++s) {
                const int b = (s & 1) ? 0 : (s & 2) ? 1 : 2;
                add(2 + b);
                e ^= 4 << b;
                T[8 * e + tt] = make_ulonglong2(v0, v1);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < RLEAF_RPT; ++u) {
            const int64_t i = tid + (int64_t)u * RLEAF_THREADS;
            if (i >= r0 + nt) continue;
            ulonglong2 x = Xs[i];
            const uint64_t ir = rotr64(ix[u], rot);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int e = (int)((ir >> (8 * k)) & 255u);
                const ulonglong2 tv = T[8 * e + ((k + lane) & 7)];
                x.x ^= tv.x;
                x.y ^= tv.y;
            }
            Xs[i] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < RLEAF_RPT; ++u) {
        const int64_t i = tid + (int64_t)u * RLEAF_THREADS;
        if (i < nrow) {
            const ulonglong2 x = Xs[i];
            X[i * ld] = x.x;
            if (two) X[i * ld + 1] = x.y;
        }
    }
}

cudaError_t launch_rref_leaf(cudaStream_t st, uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *Xb,
                             int64_t kw, const int64_t *Qb, uint64_t *Lp, int64_t w_lo, int64_t w_hi, bool prep)
{
    if (kb <= 0 || kb > RREF_LEAF_MAX || w_lo >= w_hi) return cudaSuccess;
    if (prep) {
        const cudaError_t e = launch_kernel(rref_leaf_prep_kernel, dim3((int)((kb + 63) / 64)), dim3(LEAF_THREADS), 0,
                                            st, Xb, kw, kb, Lp);
        if (e != cudaSuccess) return e;
    }
    const uint64_t *Lpc = Lp;
    return launch_kernel(rref_leaf_kernel, dim3((unsigned)((w_hi - w_lo + 1) / 2)), dim3(RLEAF_THREADS),
                         (size_t)kb * sizeof(ulonglong2), st, A, ld, row0, kb, Lpc, Qb, w_lo, w_hi);
}

constexpr int PERM_CHUNK = 8;                          // words per CTA
constexpr int PERM_THREADS = 256;

// Apply the row moves of stripes [s0, s1) to the words [w_lo, W): in stripe
// order, every staged row k of a stripe takes the words of its source row
// S_src[k] (positions before that stripe's swaps) at position r + S_off[k].
// Each CTA owns PERM_CHUNK words of every row, so CTAs never share data.
__global__ void __launch_bounds__(PERM_THREADS)
permute_trailing_kernel(uint64_t *A, int64_t ld, const StripeDesc *descs, int s0, int s1, int64_t w_lo, int64_t W,
                        const int32_t *composed)
{
    pdl_wait();
    pdl_trigger();
    if (composed && *composed >= 0) return;            // the composed form did the work
    __shared__ uint64_t tmp[SMAX][PERM_CHUNK];
    const int64_t wb = w_lo + (int64_t)blockIdx.x * PERM_CHUNK;
    if (wb >= W) return;
    const int tid = threadIdx.x;
    for (int s = s0; s < s1; ++s) {
        const StripeDesc *d = descs + s;
        const int nS = d->rbar > 0 ? d->nS : 0;
        for (int e = tid; e < nS * PERM_CHUNK; e += blockDim.x) {
            const int k = e / PERM_CHUNK, x = e - k * PERM_CHUNK;
            const int64_t w = wb + x;
            if (w < W) tmp[k][x] = A[d->S_src[k] * ld + w];
        }
        __syncthreads();
        for (int e = tid; e < nS * PERM_CHUNK; e += blockDim.x) {
            const int k = e / PERM_CHUNK, x = e - k * PERM_CHUNK;
            const int64_t w = wb + x;
            if (w < W) A[(d->r + d->S_off[k]) * ld + w] = tmp[k][x];
        }
        __syncthreads();
    }
}

// The composed form: one CTA follows every staged move of the stripes in
// order on a map tau from positions to the rows their content comes from,
// kept in shared memory for the positions r0 .. r0 + span - 1, then lists
// the positions whose content changed.  A gather of the listed source rows
// into a buffer and a scatter back apply the whole permutation to the words
// [w_lo, W) in two passes, instead of one pass per stripe.  The window path
// of the panel keeps every destination within 128 rows of the stripe's rank
// (inside the span); the block-wide path may swap with a row anywhere below.
// A destination beyond the span marks the composition failed (count -1,
// nothing written outside the span), and the per-stripe kernel launched
// after it then does the work instead.  A source beyond the span that was
// never a destination still holds its own content.
constexpr int COMPOSE_THREADS = 1024;
constexpr size_t COMPOSE_MAX_SMEM = 200 * 1024;

__global__ void __launch_bounds__(COMPOSE_THREADS)
compose_moves_kernel(const StripeDesc *descs, int s0, int s1, int64_t r0, int span, int64_t *moves, int32_t *count)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ int32_t tau[];                   // tau[p]: source offset (from r0) of position r0 + p
    __shared__ int sN, sFail;
    const int tid = threadIdx.x;
    for (int p = tid; p < span; p += COMPOSE_THREADS) tau[p] = p;
    if (tid == 0) {
        sN = 0;
        sFail = 0;
    }
    // this thread's move in a stripe (staged row tid), read one stripe ahead
    auto load = [&](int s, int64_t &dst, int64_t &src) {
        dst = -1;
        src = 0;
        if (s < s1) {
            const StripeDesc *d = descs + s;
            const int nS = d->rbar > 0 ? d->nS : 0;
            if (tid < nS) {
                src = d->S_src[tid] - r0;
                dst = d->r + d->S_off[tid] - r0;
            }
        }
    };
    int64_t dst, dn, src, sn;
    load(s0, dst, src);
    __syncthreads();
    for (int s = s0; s < s1; ++s) {
        load(s + 1, dn, sn);
        int32_t val = 0;
        if (dst >= 0) val = (src >= 0 && src < span) ? tau[src] : (int32_t)src;
        __syncthreads();                               // every move of the stripe reads before any writes
        if (dst >= 0) {
            if (dst < span) tau[dst] = val;
            else sFail = 1;
        }
        __syncthreads();
        dst = dn;
        src = sn;
    }
    if (sFail) {
        if (tid == 0) *count = -1;
        return;
    }
    for (int p = tid; p < span; p += COMPOSE_THREADS) {
        const int32_t t = tau[p];
        if (t != p) {
            const int i = atomicAdd(&sN, 1);
            moves[2 * i] = r0 + p;
            moves[2 * i + 1] = r0 + t;
        }
    }
    __syncthreads();
    if (tid == 0) *count = sN;
}

// One warp per listed move: the source row's words [w_lo, w_lo + width)
// into row i of buf (gather), or buf's row i to the destination (scatter).
template <bool GATHER>
__global__ void apply_moves_kernel(uint64_t *A, int64_t ld, const int64_t *moves, const int32_t *count, int64_t w_lo,
                                   int64_t width, uint64_t *buf)
{
    pdl_wait();
    pdl_trigger();
    const int K = *count;
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < K; i += (int64_t)gridDim.x * wpb) {
        uint64_t *row = A + moves[2 * i + (GATHER ? 1 : 0)] * ld + w_lo;
        uint64_t *b = buf + i * width;
        for (int64_t w = lane; w < width; w += 32) {
            if (GATHER) b[w] = row[w];
            else row[w] = b[w];
        }
    }
}

cudaError_t setup_blocked_kernels()
{
    const int leaf_smem = (int)(TRSM_LEAF_MAX * sizeof(ulonglong2));
    cudaError_t e = cudaFuncSetAttribute(trsm_leaf_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(trsm_leaf_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(trsm_leaf_kernel<LEAF_RPT_MAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rref_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(RREF_LEAF_MAX * sizeof(ulonglong2)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(compose_moves_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)COMPOSE_MAX_SMEM);
}

size_t permute_scratch_bytes(int s0, int s1, int64_t m, int64_t r0, int64_t w_lo, int64_t W)
{
    const int64_t span = std::min<int64_t>(m - r0, (int64_t)KS * (s1 - s0) + SMAX);
    if (span <= 0 || (size_t)span * sizeof(int32_t) > COMPOSE_MAX_SMEM || W <= w_lo) return 0;
    return (size_t)span * (2 * sizeof(int64_t) + (size_t)(W - w_lo) * sizeof(uint64_t)) + 256;
}

cudaError_t launch_permute_trailing(cudaStream_t st, uint64_t *A, int64_t ld, const StripeDesc *descs, int s0,
                                    int s1, int64_t w_lo, int64_t W, int64_t m, int64_t r0, char *scratch,
                                    size_t scratch_bytes, int num_sms)
{
    if (W <= w_lo || s1 <= s0) return cudaSuccess;
    const int64_t span = std::min<int64_t>(m - r0, (int64_t)KS * (s1 - s0) + SMAX);
    const size_t need = permute_scratch_bytes(s0, s1, m, r0, w_lo, W);
    const int64_t pblocks = (W - w_lo + PERM_CHUNK - 1) / PERM_CHUNK;
    if (need == 0 || scratch == nullptr || scratch_bytes < need || m - r0 > INT32_MAX) {
        // one pass per stripe
        return launch_kernel(permute_trailing_kernel, dim3((int)pblocks), dim3(PERM_THREADS), 0, st, A, ld, descs, s0,
                             s1, w_lo, W, (const int32_t *)nullptr);
    }
    int32_t *count = reinterpret_cast<int32_t *>(scratch);
    int64_t *moves = reinterpret_cast<int64_t *>(scratch + 256);
    uint64_t *buf = reinterpret_cast<uint64_t *>(moves + 2 * span);
    cudaError_t e = launch_kernel(compose_moves_kernel, dim3(1), dim3(COMPOSE_THREADS), (size_t)span * sizeof(int32_t),
                                  st, descs, s0, s1, r0, (int)span, moves, count);
    if (e != cudaSuccess) return e;
    const int grid = 8 * num_sms;
    e = launch_kernel(apply_moves_kernel<true>, dim3(grid), dim3(256), 0, st, A, ld, (const int64_t *)moves,
                      (const int32_t *)count, w_lo, W - w_lo, buf);
    if (e != cudaSuccess) return e;
    e = launch_kernel(apply_moves_kernel<false>, dim3(grid), dim3(256), 0, st, A, ld, (const int64_t *)moves,
                      (const int32_t *)count, w_lo, W - w_lo, buf);
    if (e != cudaSuccess) return e;
    // a composition that failed (count -1) leaves the moves to the per-stripe kernel
    return launch_kernel(permute_trailing_kernel, dim3((int)pblocks), dim3(PERM_THREADS), 0, st, A, ld, descs, s0, s1,
                         w_lo, W, (const int32_t *)count);
}

}  // namespace gf2
