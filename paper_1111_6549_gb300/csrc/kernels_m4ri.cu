// kernels_m4ri.cu -- the stripe preparation of M4RI (Algorithm 8, the
// "Method of the Four Russians Inversion"): reduced row echelon form in one
// sweep over the columns.
//
// Per 64-column stripe the panel kernel finds the pivots below the current
// rank r exactly as for PLE (Algorithm 1's rule, the rows exchanged by
// swaps).  Algorithm 8 then needs the stripe's pivot rows in reduced form --
// GaussSubmatrix clears every pivot column inside the strip -- and every
// other row, above and below, clears its bits in those columns with one table
// lookup (MakeTable + AddRowsFromTable on rows 0 .. m).  Here:
//   * the reduced pivot rows G = U11^-1 L11^-1 S, with S the raw pivot rows,
//     L11 the panel's elimination coefficients and U11 the echelon block on
//     its pivot columns, so G is the identity on the pivot columns;
//   * the rows that the swaps moved are staged into S (the update reads them
//     from there);
//   * each row's table index: the stripe word of the row that ends at its
//     position, whose bits on the pivot columns select the generators.
// Every row at a position >= r has only zeros left of the stripe (earlier
// stripes cleared them), so everything here works on the words >= the
// stripe's word.
#include "common.cuh"

#include <algorithm>

namespace gf2 {

constexpr int M4P_THREADS = 256;

__global__ void __launch_bounds__(M4P_THREADS)
m4ri_prep_kernel(const uint64_t *A, int64_t ld, int64_t W, int s, const StripeDesc *descs, const int32_t *map,
                 uint64_t *S, int64_t ldS, uint64_t *G, uint64_t *IDX, int64_t m, int nbg, int nbs)
{
    pdl_wait();
    pdl_trigger();
    const StripeDesc *d = descs + s;
    const int rbar = d->rbar;
    if (rbar == 0) return;
    const int64_t r = d->r;
    const int64_t cw = d->c >> 6;
    const int tid = threadIdx.x;
    const int bid = blockIdx.x;
    if (bid >= nbg + nbs) {
        // table index of every row: the stripe word of the row ending there
        const int64_t stride = (int64_t)(gridDim.x - nbg - nbs) * blockDim.x;
        for (int64_t i = (int64_t)(bid - nbg - nbs) * blockDim.x + tid; i < m; i += stride) {
            int64_t src = i;
            if (i >= r && i - r <= d->maxpos) {
                const int mv = map[i];
                if (mv >= 0 && (mv >> 8) == s) src = d->S_src[mv & 255];
            }
            IDX[i] = A[src * ld + cw];
        }
        return;
    }
    if (bid >= nbg) {
        // the rows displaced by the swaps, words [cw, W)
        for (int k = rbar + (bid - nbg); k < d->nS; k += nbs) {
            const uint64_t *src = A + d->S_src[k] * ld;
            uint64_t *dst = S + (int64_t)k * ldS;
            for (int64_t w = cw + tid; w < W; w += blockDim.x) dst[w] = src[w];
        }
        return;
    }
    // reduced pivot rows: G = (U11^-1 L11^-1) S over words [cw, W)
    __shared__ uint64_t sM[KS];
    __shared__ uint64_t sIn[KS][4];
    __shared__ int64_t sSrc[KS];
    if (tid < rbar) {
        uint64_t acc = 0;
        const uint64_t mp = d->Minv[tid];
        for (int q = 0; q < rbar; ++q)
            if ((mp >> q) & 1ull) acc ^= d->Linv[q];
        sM[tid] = acc;
        sSrc[tid] = d->S_src[tid];
    }
    __syncthreads();
    const int p = tid >> 2, wq = tid & 3;
    for (int64_t wb = cw + (int64_t)bid * 4; wb < W; wb += (int64_t)nbg * 4) {
        const int64_t w = wb + wq;
        sIn[p][wq] = (p < rbar && w < W) ? A[sSrc[p] * ld + w] : 0ull;
        __syncthreads();
        if (p < rbar && w < W) {
            const uint64_t mrow = sM[p];
            uint64_t acc = 0;
            for (int q = 0; q < rbar; ++q)
                if ((mrow >> q) & 1ull) acc ^= sIn[q][wq];
            G[(int64_t)p * ldS + w] = acc;
        }
        __syncthreads();
    }
}

cudaError_t launch_m4ri_prep(cudaStream_t st, const uint64_t *A, int64_t ld, int64_t W, int s,
                             const StripeDesc *descs, const int32_t *map, uint64_t *S, int64_t ldS, uint64_t *G,
                             uint64_t *IDX, int64_t m, int num_sms)
{
    const int nbg = (int)std::min<int64_t>(num_sms, (W + 3) / 4);
    const int nbs = 16;
    int nbi = (int)std::min<int64_t>(2 * num_sms, (m + M4P_THREADS - 1) / M4P_THREADS);
    if (nbi < 1) nbi = 1;
    return launch_kernel(m4ri_prep_kernel, dim3(nbg + nbs + nbi), dim3(M4P_THREADS), 0, st, A, ld, W, s, descs, map, S,
                         ldS, G, IDX, m, nbg, nbs);
}

}  // namespace gf2
