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
// buffer (the GEMM and TRSM operands), trsm_diag_kernel applies the inverse
// of one 64 x 64 unit lower diagonal block of L11 to its 64 rows; the rest is
// the table update (UPD_MUL) and gf2_mul.
#include "panel_dev.cuh"

namespace gf2 {

// out[i][w] = bits [c0 + 64 w, c0 + 64 w + 64) of row row0 + i, masked to the
// first kb bits (i < rows, w < kw)
__global__ void gather_lbits_kernel(const uint64_t *__restrict__ A, int64_t ld, int64_t W, int64_t row0,
                                    int64_t rows, int64_t c0, int64_t kb, int64_t kw, uint64_t *__restrict__ out)
{
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
    gather_lbits_kernel<<<(int)blocks, 256, 0, st>>>(A, ld, W, row0, rows, c0, kb, kw, out);
    return cudaGetLastError();
}

// out[i][w] = the bits of row row0 + i at the columns Qb[64 w .. 64 w + 64)
// (bit b of word w from column Qb[64 w + b]) for the first kb entries of the
// increasing column list Qb (i < rows, w < kw).  A word whose 64 columns are
// consecutive is one shifted load; the others go bit by bit.
__global__ void gather_pivbits_kernel(const uint64_t *__restrict__ A, int64_t ld, int64_t W, int64_t row0,
                                      int64_t rows, const int64_t *__restrict__ Qb, int64_t kb, int64_t kw,
                                      uint64_t *__restrict__ out)
{
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
    gather_pivbits_kernel<<<(int)blocks, 256, 0, st>>>(A, ld, W, row0, rows, Qb, kb, kw, out);
    return cudaGetLastError();
}

constexpr int TRSM_THREADS = 256;

// Rows X[0 .. nt) (X = A + row0 * ld) <- Linv X over the words [w_lo, W),
// Linv the inverse of the unit lower nt x nt block whose strictly lower bits
// are Lblk[p] (word t of the gathered L rows 64 t + p).
__global__ void __launch_bounds__(TRSM_THREADS)
trsm_diag_kernel(uint64_t *A, int64_t ld, int64_t row0, int nt, const uint64_t *__restrict__ Lt, int64_t ldt,
                 int64_t t, int64_t w_lo, int64_t W)
{
    __shared__ uint64_t sL[KS], sM[KS];
    __shared__ uint64_t sIn[KS][4];
    const int tid = threadIdx.x;
    if (tid < KS) sL[tid] = (tid < nt) ? (Lt[(64 * t + tid) * ldt + t] & ((1ull << tid) - 1ull)) : 0ull;
    __syncthreads();
    if (tid < 32) warp_lower_inverse(sL, nt, sM);
    __syncthreads();
    const int p = tid >> 2, wq = tid & 3;
    for (int64_t wb = w_lo + (int64_t)blockIdx.x * 4; wb < W; wb += (int64_t)gridDim.x * 4) {
        const int64_t w = wb + wq;
        sIn[p][wq] = (p < nt && w < W) ? A[(row0 + p) * ld + w] : 0ull;
        __syncthreads();
        if (p < nt && w < W) {
            const uint64_t mrow = sM[p];
            uint64_t acc = 0;
            for (int q = 0; q < nt; ++q)
                if ((mrow >> q) & 1ull) acc ^= sIn[q][wq];
            A[(row0 + p) * ld + w] = acc;
        }
        __syncthreads();
    }
}

cudaError_t launch_trsm_diag(cudaStream_t st, uint64_t *A, int64_t ld, int64_t row0, int nt, const uint64_t *Lt,
                             int64_t ldt, int64_t t, int64_t w_lo, int64_t W, int num_sms)
{
    int64_t blocks = (W - w_lo + 3) / 4;
    if (blocks > 2 * num_sms) blocks = 2 * num_sms;
    if (blocks < 1) blocks = 1;
    trsm_diag_kernel<<<(int)blocks, TRSM_THREADS, 0, st>>>(A, ld, row0, nt, Lt, ldt, t, w_lo, W);
    return cudaGetLastError();
}

constexpr int PERM_CHUNK = 8;                          // words per CTA
constexpr int PERM_THREADS = 256;

// Apply the row moves of stripes [s0, s1) to the words [w_lo, W): in stripe
// order, every staged row k of a stripe takes the words of its source row
// S_src[k] (positions before that stripe's swaps) at position r + S_off[k].
// Each CTA owns PERM_CHUNK words of every row, so CTAs never share data.
__global__ void __launch_bounds__(PERM_THREADS)
permute_trailing_kernel(uint64_t *A, int64_t ld, const StripeDesc *descs, int s0, int s1, int64_t w_lo, int64_t W)
{
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

cudaError_t launch_permute_trailing(cudaStream_t st, uint64_t *A, int64_t ld, const StripeDesc *descs, int s0,
                                    int s1, int64_t w_lo, int64_t W)
{
    const int64_t blocks = (W - w_lo + PERM_CHUNK - 1) / PERM_CHUNK;
    if (blocks <= 0 || s1 <= s0) return cudaSuccess;
    permute_trailing_kernel<<<(int)blocks, PERM_THREADS, 0, st>>>(A, ld, descs, s0, s1, w_lo, W);
    return cudaGetLastError();
}

}  // namespace gf2
