// kernels_rref.cu -- RREF recovery from the PLE form, and solve helpers.
//
// Section 5 computes the RREF by first computing the PLE decomposition and
// then recovering the reduced form from it (the recovery is not spelled out).
// Here: drop L (every row keeps only its columns >= its own index; rows past
// the rank become zero), then walk the pivot blocks of the PLE stripes from
// the last to the first.  For block s (rows r_s .. r_s+rbar-1, pivot columns
// inside [c_s, c_s+64)):
//   1. reduce the block against itself: rows <- U11^-1 rows, U11 = the block
//      restricted to its pivot columns (unit upper triangular), so each
//      pivot column becomes a unit vector inside the block;
//   2. clear the block's pivot columns in every row above the block with the
//      tabulated update (kernels_update.cu, UPD_RREF), indexed by the row's
//      stripe word, which rref_prep copies out before the update starts.
// Later blocks only touch columns >= c_s + 64, so the stripe word of block s
// still equals the E11 recorded by the panel when block s is processed.
#include "common.cuh"

namespace gf2 {

__global__ void rref_lclear_kernel(uint64_t *A, int64_t m, int64_t W, int64_t ld, const int64_t *r_dev)
{
    pdl_wait();
    pdl_trigger();
    const int64_t r = *r_dev;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp0; i < m; i += nwarps) {
        uint64_t *row = A + i * ld;
        if (i < r) {
            const int64_t wl = i >> 6;
            for (int64_t w = lane; w < wl; w += 32) row[w] = 0;
            if (lane == 0 && (i & 63)) row[wl] &= ~((1ull << (i & 63)) - 1ull);
        } else {
            for (int64_t w = lane; w < W; w += 32) row[w] = 0;
        }
    }
}

cudaError_t launch_rref_lclear(cudaStream_t st, uint64_t *A, int64_t m, int64_t W, int64_t ld,
                               const int64_t *r_dev, int num_sms)
{
    int64_t blocks = (m * 32 + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 8 * num_sms) blocks = 8 * num_sms;
    return launch_kernel(rref_lclear_kernel, dim3((int)blocks), dim3(256), 0, st, A, m, W, ld, r_dev);
}

constexpr int RPREP_THREADS = 256;

__global__ void __launch_bounds__(RPREP_THREADS)
rref_prep_kernel(uint64_t *A, int64_t ld, int64_t W, int s, const StripeDesc *descs, uint64_t *IDX,
                 int nbr)
{
    pdl_wait();
    pdl_trigger();
    const StripeDesc *d = descs + s;
    const int rbar = d->rbar;
    if (rbar == 0) return;
    const int64_t r = d->r;
    const int64_t cw = d->c >> 6;
    if ((int)blockIdx.x >= nbr) {
        // stripe words of the rows above the block: the update's table index
        const int64_t stride = (int64_t)(gridDim.x - nbr) * blockDim.x;
        for (int64_t i = (int64_t)(blockIdx.x - nbr) * blockDim.x + threadIdx.x; i < r; i += stride)
            IDX[i] = A[i * ld + cw];
        return;
    }
    __shared__ uint64_t sM[KS];
    __shared__ uint64_t sIn[KS][4];
    const int tid = threadIdx.x;
    // U11^-1 was computed once by the PLE's prep kernel
    for (int p = tid; p < rbar; p += blockDim.x) sM[p] = d->Minv[p];
    __syncthreads();
    // rows <- U11^-1 rows over words [cw, W), four words per step
    const int p = tid >> 2, wq = tid & 3;
    for (int64_t wb = cw + (int64_t)blockIdx.x * 4; wb < W; wb += (int64_t)nbr * 4) {
        const int64_t w = wb + wq;
        sIn[p][wq] = (p < rbar && w < W) ? A[(r + p) * ld + w] : 0ull;
        __syncthreads();
        if (p < rbar && w < W) {
            const uint64_t mrow = sM[p];
            uint64_t acc = 0;
            for (int q = 0; q < rbar; ++q) acc ^= sIn[q][wq] & (0ull - ((mrow >> q) & 1ull));
            A[(r + p) * ld + w] = acc;
        }
        __syncthreads();
    }
}

cudaError_t launch_rref_prep(cudaStream_t st, uint64_t *A, int64_t ld, int64_t W, int s,
                             const StripeDesc *descs, uint64_t *IDX, int64_t m, int num_sms)
{
    // block-reduce CTAs: enough to cover the words right of the stripe start
    // (an upper bound: the stripe start is only known on the device)
    int64_t nbr = (W + 3) / 4;
    if (nbr > 2 * num_sms) nbr = 2 * num_sms;
    if (nbr < 1) nbr = 1;
    int64_t nidx = (m + RPREP_THREADS - 1) / RPREP_THREADS;
    if (nidx > 2 * num_sms) nidx = 2 * num_sms;
    if (nidx < 1) nidx = 1;
    return launch_kernel(rref_prep_kernel, dim3((int)(nbr + nidx)), dim3(RPREP_THREADS), 0, st, A, ld, W, s, descs, IDX,
                         (int)nbr);
}

// Bookends of a block of fused RREF passes (see UpdArgs::rref_fused): the
// first pass's table index (the stripe word of the rows above it) and, after
// the last pass, its reduced pivot rows from the buffer into A.
__global__ void rref_aux_kernel(uint64_t *A, int64_t ld, const StripeDesc *flush_desc, const uint64_t *gbuf,
                                int64_t ldg, int64_t W, int64_t skip_lo, int64_t skip_hi,
                                const StripeDesc *snap_desc, uint64_t *idx, int64_t row_lo)
{
    pdl_wait();
    pdl_trigger();
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    if (flush_desc) {
        const int rbar = flush_desc->rbar;
        const int64_t c0 = flush_desc->c >> 6;
        const int64_t nw = W - c0;
        if (rbar > 0 && nw > 0)
            for (int64_t e = gt; e < rbar * nw; e += gs) {
                const int64_t t = e / nw, word = c0 + (e - t * nw);
                if (word >= skip_lo && word < skip_hi) continue;
                A[(flush_desc->r + t) * ld + word] = gbuf[t * ldg + word];
            }
    }
    if (snap_desc) {
        const int64_t cw = snap_desc->c >> 6;
        for (int64_t i = row_lo + gt; i < snap_desc->r; i += gs) idx[i] = A[i * ld + cw];
    }
}

cudaError_t launch_rref_aux(cudaStream_t st, uint64_t *A, int64_t ld, const StripeDesc *flush_desc,
                            const uint64_t *gbuf, int64_t ldg, int64_t W, int64_t skip_lo, int64_t skip_hi,
                            const StripeDesc *snap_desc, uint64_t *idx, int64_t row_lo, int num_sms)
{
    return launch_kernel(rref_aux_kernel, dim3(2 * num_sms), dim3(256), 0, st, A, ld, flush_desc, gbuf, ldg, W,
                         skip_lo, skip_hi, snap_desc, idx, row_lo);
}

__global__ void copy_rank_kernel(const int64_t *r_dev, int64_t *rank_dev)
{
    pdl_wait();
    pdl_trigger();
    *rank_dev = *r_dev;
}

cudaError_t launch_copy_rank(cudaStream_t st, const int64_t *r_dev, int64_t *rank_dev)
{
    return launch_kernel(copy_rank_kernel, dim3(1), dim3(1), 0, st, r_dev, rank_dev);
}

// ---- solve: consistency of the transformed right-hand side, then X

// flag <- 1 when some row >= rank of the right-hand-side words is nonzero
__global__ void solve_check_kernel(const uint64_t *Aug, int64_t ldaug, int64_t n, int64_t wa,
                                   int64_t wb, const int64_t *r_dev, int32_t *flag)
{
    const int64_t r = *r_dev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (n - r) * wb; t += stride) {
        const int64_t i = r + t / wb, w = t % wb;
        if (Aug[i * ldaug + wa + w]) atomicExch(flag, 1);
    }
}

// B <- 0
__global__ void solve_zero_kernel(uint64_t *B, int64_t ldb, int64_t n, int64_t wb)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * wb; t += stride)
        B[(t / wb) * ldb + (t % wb)] = 0;
}

// X[Q[p]] <- reduced right-hand side of pivot row p
__global__ void solve_scatter_kernel(const uint64_t *Aug, int64_t ldaug, int64_t wa, int64_t wb,
                                     const int64_t *r_dev, const int64_t *Q, uint64_t *B, int64_t ldb)
{
    const int64_t r = *r_dev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < r * wb; t += stride) {
        const int64_t p = t / wb, w = t % wb;
        B[Q[p] * ldb + w] = Aug[p * ldaug + wa + w];
    }
}

cudaError_t launch_solve_check(cudaStream_t st, const uint64_t *Aug, int64_t ldaug, int64_t n,
                               int64_t wa, int64_t wb, const int64_t *r_dev, int32_t *flag)
{
    int64_t blocks = (n * wb + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    solve_check_kernel<<<(int)blocks, 256, 0, st>>>(Aug, ldaug, n, wa, wb, r_dev, flag);
    return cudaGetLastError();
}

cudaError_t launch_solve_finish(cudaStream_t st, const uint64_t *Aug, int64_t ldaug, int64_t n,
                                int64_t wa, int64_t wb, const int64_t *r_dev, const int64_t *Q,
                                uint64_t *B, int64_t ldb)
{
    int64_t blocks = (n * wb + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    solve_zero_kernel<<<(int)blocks, 256, 0, st>>>(B, ldb, n, wb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    solve_scatter_kernel<<<(int)blocks, 256, 0, st>>>(Aug, ldaug, wa, wb, r_dev, Q, B, ldb);
    return cudaGetLastError();
}

__global__ void solve_status_kernel(const int64_t *r_dev, const int32_t *flag, int64_t n, int32_t *status)
{
    *status = *flag ? 2 : (*r_dev == n ? 0 : 1);
}

cudaError_t launch_solve_status(cudaStream_t st, const int64_t *r_dev, const int32_t *flag, int64_t n,
                                int32_t *status)
{
    solve_status_kernel<<<1, 1, 0, st>>>(r_dev, flag, n, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Compact recovery: the reduced rows written back.  Row i < r is the
// identity on the pivot columns (its own pivot Q[i] set, every other pivot
// column clear) and, on the non-pivot columns, the reduced bits C[i]
// (kwn words; compact position s holds the s-th non-pivot column).
// npmask[w]: the non-pivot columns of word w; npstart[w]: the compact
// position of the first of them.  Every word of rows < r is written.
__global__ void rref_scatter_kernel(uint64_t *A, int64_t ld, int64_t W, int64_t r, const int64_t *__restrict__ Q,
                                    const uint64_t *__restrict__ C, int64_t kwn,
                                    const uint64_t *__restrict__ npmask, const int64_t *__restrict__ npstart)
{
    pdl_wait();
    pdl_trigger();
    const int64_t total = r * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / W, w = t - i * W;
        const int64_t qi = __ldg(Q + i);
        uint64_t word = (qi >> 6) == w ? (1ull << (qi & 63)) : 0ull;
        const uint64_t mask = __ldg(npmask + w);
        if (mask) {
            const int nb = __popcll(mask);
            const int64_t s0 = __ldg(npstart + w);
            const uint64_t *ci = C + i * kwn;
            const int64_t cw = s0 >> 6;
            const int off = (int)(s0 & 63);
            uint64_t f = ci[cw] >> off;
            if (off && off + nb > 64) f |= ci[cw + 1] << (64 - off);
            if (nb < 64) f &= (1ull << nb) - 1ull;
            if (nb == 64) {
                word = f;                                // no pivot column in this word
            } else if (nb <= 32) {
                // deposit the bits of f, lowest first, at the set positions of mask
                uint64_t m2 = mask;
                while (m2) {
                    const uint64_t low = m2 & (~m2 + 1ull);
                    if (f & 1ull) word |= low;
                    f >>= 1;
                    m2 ^= low;
                }
            } else {
                // the same by opening a zero at every clear position of mask
                uint64_t z = ~mask;
                while (z) {
                    const int p = __ffsll((long long)z) - 1;
                    const uint64_t lowp = (1ull << p) - 1ull;
                    f = p == 63 ? (f & lowp) : ((f & lowp) | ((f >> p) << (p + 1)));
                    z &= z - 1ull;
                }
                word |= f;
            }
        }
        A[i * ld + w] = word;
    }
}

cudaError_t launch_rref_scatter(cudaStream_t st, uint64_t *A, int64_t ld, int64_t W, int64_t r, const int64_t *Q,
                                const uint64_t *C, int64_t kwn, const uint64_t *npmask, const int64_t *npstart,
                                int num_sms)
{
    int64_t blocks = (r * W + 255) / 256;
    if (blocks < 1) return cudaSuccess;
    if (blocks > 16 * num_sms) blocks = 16 * num_sms;
    return launch_kernel(rref_scatter_kernel, dim3((int)blocks), dim3(256), 0, st, A, ld, W, r, Q, C, kwn, npmask,
                         npstart);
}

// ---------------------------------------------------------------------------
constexpr int JN_MAXC = 8;                 // non-pivot columns the narrow join takes
constexpr int JN_THREADS = 512;
constexpr size_t JN_MAX_SMEM = 48 * 1024;  // the columns' bit vectors in shared memory

static size_t join_narrow_smem(int64_t kwx, int nnp) { return (size_t)nnp * (size_t)kwx * sizeof(uint64_t); }

bool join_narrow_fits(int64_t kwx, int64_t nnp)
{
    return nnp >= 1 && nnp <= JN_MAXC && join_narrow_smem(kwx, (int)nnp) <= JN_MAX_SMEM;
}

// A join of the compact recovery when at most JN_MAXC columns have no pivot:
// C1 ^= X C2 with X (rows x kx bits, kwx words per row), C2 (kx rows of one
// word, bits 0 .. nnp-1) and C1 (rows of one word).  Each CTA first turns C2
// into nnp bit columns over its kx rows in shared memory (one ballot per 32
// rows and column); a warp per row of X then takes, per column, the parity
// of the row AND the column, and the row's word gets the parities.  Reads X
// once, with no operand expansion.
__global__ void __launch_bounds__(JN_THREADS)
join_narrow_kernel(uint64_t *__restrict__ C1, const uint64_t *__restrict__ X, int64_t kwx,
                   const uint64_t *__restrict__ C2, int64_t kx, int nnp, int64_t rows)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint64_t colv[];   // [c][w]: bit k % 64 of word k / 64 = bit c of C2[k]
    uint32_t *colv32 = reinterpret_cast<uint32_t *>(colv);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = JN_THREADS / 32;
    const unsigned FULL = 0xffffffffu;
    const int64_t groups = 2 * kwx;                       // 32-row groups, whole words
    for (int64_t g = warp; g < groups; g += NW) {
        const int64_t k = 32 * g + lane;
        const uint64_t v = k < kx ? C2[k] : 0ull;
        for (int c = 0; c < nnp; ++c) {
            const unsigned b = __ballot_sync(FULL, (unsigned)(v >> c) & 1u);
            if (lane == 0) colv32[(int64_t)c * groups + g] = b;
        }
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * NW + warp; i < rows; i += (int64_t)gridDim.x * NW) {
        const uint64_t *xr = X + i * kwx;
        uint32_t par = 0;                                 // bit c: this lane's share of column c's parity
        for (int64_t w = lane; w < kwx; w += 32) {
            const uint64_t xw = xr[w];
            for (int c = 0; c < nnp; ++c) par ^= (uint32_t)(__popcll(xw & colv[(int64_t)c * kwx + w]) & 1) << c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) par ^= __shfl_xor_sync(FULL, par, o);
        if (lane == 0 && par) C1[i] ^= (uint64_t)par;
    }
}

cudaError_t launch_join_narrow(cudaStream_t st, uint64_t *C1, const uint64_t *X, int64_t kwx, const uint64_t *C2,
                               int64_t kx, int nnp, int64_t rows, int num_sms)
{
    if (rows <= 0 || kx <= 0 || nnp <= 0) return cudaSuccess;
    if (!join_narrow_fits(kwx, nnp)) return cudaErrorInvalidValue;
    int64_t blocks = (rows + JN_THREADS / 32 - 1) / (JN_THREADS / 32);
    if (blocks > 2 * num_sms) blocks = 2 * num_sms;
    return launch_kernel(join_narrow_kernel, dim3((int)blocks), dim3(JN_THREADS), join_narrow_smem(kwx, nnp), st, C1,
                         X, kwx, C2, kx, nnp, rows);
}

}  // namespace gf2
