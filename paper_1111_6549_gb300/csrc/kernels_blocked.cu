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
// Fused TRSM leaf: X <- L^-1 X for the kb <= TRSM_LEAF_ROWS rows X = A[row0 ..
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
// the leaf's rows (at most TRSM_LEAF_ROWS x 16 bytes) stay in shared memory
// for all steps: loaded once, updated in place, stored once.  Thread t owns
// the rows t, t + 256, ... in every step, so it loads the next step's
// indices of its rows while the current step runs.
constexpr int LEAF_RPT = (int)(TRSM_LEAF_ROWS / LEAF_THREADS);
constexpr size_t LEAF_SMEM = (size_t)TRSM_LEAF_ROWS * 2 * sizeof(uint64_t);

__global__ void __launch_bounds__(LEAF_THREADS)
trsm_leaf_kernel(uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *__restrict__ Lp, int64_t w_lo,
                 int64_t W)
{
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) uint64_t T[8 * 256 * 2];      // eight 8-bit tables of 16-byte entries
    __shared__ uint64_t G[KS][2];
    extern __shared__ __align__(16) uint64_t Xs[];       // [row][2]: the CTA's two words of the leaf's rows
    const int tid = threadIdx.x;
    const int64_t w0 = w_lo + 2 * (int64_t)blockIdx.x;
    if (w0 >= W) return;
    const bool two = w0 + 1 < W;
    uint64_t *X = A + row0 * ld + w0;
    for (int u = 0; u < LEAF_RPT; ++u) {
        const int64_t i = tid + (int64_t)u * LEAF_THREADS;
        if (i < kb) {
            Xs[2 * i] = X[i * ld];
            Xs[2 * i + 1] = two ? X[i * ld + 1] : 0ull;
        }
    }
    const int nsteps = (int)((kb + 63) / 64);
    uint64_t ixn[LEAF_RPT];                                // the indices of this thread's rows, one step ahead
#pragma unroll
    for (int u = 0; u < LEAF_RPT; ++u) {
        const int64_t i = tid + (int64_t)u * LEAF_THREADS;
        ixn[u] = (i < kb) ? __ldg(Lp + i) : 0ull;
    }
    for (int t = 0; t < nsteps; ++t) {
        const int64_t r0 = 64 * (int64_t)t;
        const int nt = (int)min((int64_t)KS, kb - r0);
        __syncthreads();                                   // rows of this step written by the last one
        if (tid < 2 * KS) {
            const int p = tid >> 1, q = tid & 1;
            G[p][q] = (p < nt) ? Xs[2 * (r0 + p) + q] : 0ull;
        }
        uint64_t ix[LEAF_RPT];
#pragma unroll
        for (int u = 0; u < LEAF_RPT; ++u) {
            ix[u] = ixn[u];
            const int64_t i = tid + (int64_t)u * LEAF_THREADS;
            ixn[u] = (t + 1 < nsteps && i >= r0 + 64 && i < kb) ? __ldg(Lp + (int64_t)(t + 1) * kb + i) : 0ull;
        }
        __syncthreads();
        if (tid < 128) {
            // table tau (rows 8 tau .. 8 tau + 7), 32-entry segment sg, word q:
            // Gray-code walk from the segment's base entry
            const int q = tid & 1, sg = (tid >> 1) & 7, tau = tid >> 4;
            uint64_t g[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) g[b] = G[8 * tau + b][q];
            uint64_t val = ((sg & 1) ? g[5] : 0ull) ^ ((sg & 2) ? g[6] : 0ull) ^ ((sg & 4) ? g[7] : 0ull);
            uint64_t *Tt = T + (tau * 256 + 32 * sg) * 2 + q;
            int x = 0;
            Tt[0] = val;
#pragma unroll
            for (int i = 1; i < 32; ++i) {
                const int b = (i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : 4;
                x ^= 1 << b;
                val ^= g[b];
                Tt[x * 2] = val;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < LEAF_RPT; ++u) {
            const int64_t i = tid + (int64_t)u * LEAF_THREADS;
            if (i < r0 || i >= kb) continue;
            uint64_t x0 = Xs[2 * i], x1 = Xs[2 * i + 1];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const ulonglong2 tv =
                    *reinterpret_cast<const ulonglong2 *>(T + (b * 256 + ((ix[u] >> (8 * b)) & 255u)) * 2);
                x0 ^= tv.x;
                x1 ^= tv.y;
            }
            Xs[2 * i] = x0;
            Xs[2 * i + 1] = x1;
        }
    }
    __syncthreads();
    for (int u = 0; u < LEAF_RPT; ++u) {
        const int64_t i = tid + (int64_t)u * LEAF_THREADS;
        if (i < kb) {
            X[i * ld] = Xs[2 * i];
            if (two) X[i * ld + 1] = Xs[2 * i + 1];
        }
    }
}

cudaError_t launch_trsm_leaf(cudaStream_t st, uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *Lt,
                             int64_t ldt, uint64_t *Lp, int64_t w_lo, int64_t W)
{
    if (kb <= 0 || kb > TRSM_LEAF_ROWS || w_lo >= W) return cudaSuccess;
    cudaError_t e =
        launch_kernel(trsm_leaf_prep_kernel, dim3((int)((kb + 63) / 64)), dim3(LEAF_THREADS), 0, st, Lt, ldt, kb, Lp);
    if (e != cudaSuccess) return e;
    return launch_kernel(trsm_leaf_kernel, dim3((int)((W - w_lo + 1) / 2)), dim3(LEAF_THREADS), LEAF_SMEM, st, A, ld,
                         row0, kb, (const uint64_t *)Lp, w_lo, W);
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
    cudaError_t e = cudaFuncSetAttribute(trsm_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LEAF_SMEM);
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
