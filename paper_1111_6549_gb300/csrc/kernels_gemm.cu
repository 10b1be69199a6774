// kernels_gemm.cu -- the GF(2) product C ^= A B on the tensor cores through a
// plain library low-precision GEMM, for large inner dimensions.
//
// Over GF(2), (A B)[i][j] is the parity of the integer count
// sum_k A[i][k] B[k][j].  With every bit written as a floating-point 0 or
// 1.0, a GEMM with fp32 accumulation returns that count exactly (every
// partial sum is an integer below 2^24), and its low bit is the GF(2) entry.
// Two operand formats: FP4 E2M1 (1.0 = 0b0010, two values per byte) with
// every 16-value block scale 1.0 (UE4M3 0x38) -- the default, at the FP4
// tensor rate -- and FP8 E4M3 (1.0 = 0x38).  The library only multiplies;
// the bit work is here:
//   * expand_rows_kernel: rows of bits -> rows of FP4 / FP8 values, K-major
//     (the layout the GEMM wants for both operands);
//   * expand_transpose_kernel: B (k x n bits) -> B^T as n rows of k values,
//     transposing 64 x 64 bit blocks with warp shuffles;
//   * parity_kernel: each fp32 count -> its parity bit, 64 per word, XORed
//     into C (so C accumulates).
#include "common.cuh"

#ifdef GF2_WITH_CUBLASLT
#include <cublasLt.h>
#endif

#include <algorithm>
#include <new>

namespace gf2 {

namespace {

// 4 bits -> 4 FP8 bytes (1.0 = 0x38 where the bit is set)
__device__ __forceinline__ uint32_t nib_fp8(uint32_t b)
{
    uint32_t t = (b & 15u) * 0x01010101u;   // the nibble in every byte
    t &= 0x08040201u;                       // byte i keeps bit i
    t = ((t + 0x7F7F7F7Fu) & 0x80808080u) >> 7;   // 1 in the bytes whose bit was set
    return t * 0x38u;
}

// 64 bits -> 64 FP8 bytes at dst (16-byte aligned)
__device__ __forceinline__ void store_word_fp8(uint8_t *dst, uint64_t w)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t h = (uint32_t)(w >> (16 * q));
        uint4 v;
        v.x = nib_fp8(h);
        v.y = nib_fp8(h >> 4);
        v.z = nib_fp8(h >> 8);
        v.w = nib_fp8(h >> 12);
        *reinterpret_cast<uint4 *>(dst + 16 * q) = v;
    }
}

// 16 bits -> 16 E2M1 nibbles (bit i -> nibble i, 1.0 = 0b0010 where set)
__device__ __forceinline__ uint64_t spread16_fp4(uint64_t x)
{
    x &= 0xFFFFull;
    x = (x | (x << 24)) & 0x000000FF000000FFull;
    x = (x | (x << 12)) & 0x000F000F000F000Full;
    x = (x | (x << 6)) & 0x0303030303030303ull;
    x = (x | (x << 3)) & 0x1111111111111111ull;
    return x << 1;
}

// 64 bits -> 32 bytes of E2M1 pairs at dst (16-byte aligned)
__device__ __forceinline__ void store_word_fp4(uint8_t *dst, uint64_t w)
{
    const uint64_t q0 = spread16_fp4(w), q1 = spread16_fp4(w >> 16), q2 = spread16_fp4(w >> 32),
                   q3 = spread16_fp4(w >> 48);
    uint4 a, b;
    a.x = (uint32_t)q0;
    a.y = (uint32_t)(q0 >> 32);
    a.z = (uint32_t)q1;
    a.w = (uint32_t)(q1 >> 32);
    b.x = (uint32_t)q2;
    b.y = (uint32_t)(q2 >> 32);
    b.z = (uint32_t)q3;
    b.w = (uint32_t)(q3 >> 32);
    *reinterpret_cast<uint4 *>(dst) = a;
    *reinterpret_cast<uint4 *>(dst + 16) = b;
}

// one 64-bit word in the chosen element format: FP8 (64 bytes) or FP4 (32)
template <int FMT>
__device__ __forceinline__ void store_word(uint8_t *dst, uint64_t w)
{
    if (FMT == 8)
        store_word_fp8(dst, w);
    else
        store_word_fp4(dst, w);
}

__device__ __forceinline__ unsigned transpose32_g(unsigned x)
{
    const int lane = threadIdx.x & 31;
    const unsigned masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int j = 16 >> k;
        const unsigned m = masks[k];
        const unsigned y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? (((y >> j) & m) | (x & ~m)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

}  // namespace

// out row i = bits k0 .. k0+kp of row i (zero past k) as kp FP8 or FP4 values
template <int FMT>
__global__ void expand_rows_kernel(const uint64_t *__restrict__ A, int64_t lda, int64_t rows, int64_t k0,
                                   int64_t k, int64_t kp, uint8_t *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const int64_t rb = kp * FMT / 8;                   // bytes per output row
    const int64_t wpr = kp >> 6;                       // words per output row
    const int64_t total = rows * wpr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / wpr, w = t - i * wpr;
        const int64_t kb = k0 + 64 * w;                // first bit of this word (multiple of 64)
        uint64_t v = 0;
        if (kb < k) {
            v = A[i * lda + (kb >> 6)];
            if (k - kb < 64) v &= (1ull << (k - kb)) - 1ull;
        }
        store_word<FMT>(out + i * rb + 8 * FMT * w, v);
    }
}

// out row j = column j of B over rows k0 .. k0+kp (zero past k) as kp FP8 or
// FP4 values.  One warp per 64 x 64 bit block: lanes load rows kr and kr+32
// of the block, four 32 x 32 shuffle transposes give lane c the columns c and
// 32 + c.
template <int FMT>
__global__ void expand_transpose_kernel(const uint64_t *__restrict__ B, int64_t ldb, int64_t k0, int64_t k,
                                        int64_t n, int64_t kp, uint8_t *__restrict__ out)
{
    pdl_wait();
    pdl_trigger();
    const int64_t rb = kp * FMT / 8;
    const int lane = threadIdx.x & 31;
    const int64_t nbk = kp >> 6, nbn = (n + 63) >> 6;
    const int64_t total = nbk * nbn;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t blk = wid; blk < total; blk += nw) {
        const int64_t bk = blk / nbn, bn = blk - bk * nbn;
        const int64_t r0 = k0 + 64 * bk + lane, r1 = r0 + 32;
        const uint64_t x0 = (r0 < k) ? B[r0 * ldb + bn] : 0ull;
        const uint64_t x1 = (r1 < k) ? B[r1 * ldb + bn] : 0ull;
        const unsigned t00 = transpose32_g((unsigned)x0), t01 = transpose32_g((unsigned)(x0 >> 32));
        const unsigned t10 = transpose32_g((unsigned)x1), t11 = transpose32_g((unsigned)(x1 >> 32));
        // lane c: column 64 bn + c over the block's 64 rows, and column 64 bn + 32 + c
        const int64_t c0 = 64 * bn + lane, c1 = c0 + 32;
        if (c0 < n) store_word<FMT>(out + c0 * rb + 8 * FMT * bk, ((uint64_t)t10 << 32) | t00);
        if (c1 < n) store_word<FMT>(out + c1 * rb + 8 * FMT * bk, ((uint64_t)t11 << 32) | t01);
    }
}

// C[i][w] ^= parity bits of D[i][64 w .. 64 w + 63] (fp32 integer counts < 2^23).
// One warp per group of PAR_WORDS output words of a row: all of their
// coalesced 32-float loads are issued before the ballots.
constexpr int PAR_WORDS = 4;

__global__ void parity_kernel(const float *__restrict__ D, int64_t ldd, int64_t rows, int64_t n, uint64_t *C,
                              int64_t ldc)
{
    const int lane = threadIdx.x & 31;
    const int64_t W = (n + 63) >> 6;
    const int64_t G = (W + PAR_WORDS - 1) / PAR_WORDS;
    const int64_t total = rows * G;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = wid; t < total; t += nw) {
        const int64_t i = t / G, w0 = (t - i * G) * PAR_WORDS;
        float f[2 * PAR_WORDS];
#pragma unroll
        for (int q = 0; q < 2 * PAR_WORDS; ++q) {
            const int64_t j = 64 * w0 + 32 * q + lane;
            f[q] = (j < n) ? D[i * ldd + j] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < PAR_WORDS; ++q) {
            // adding 2^23 puts the integer count in the low mantissa bits
            const unsigned lo = __ballot_sync(0xffffffffu, __float_as_uint(f[2 * q] + 8388608.0f) & 1u);
            const unsigned hi = __ballot_sync(0xffffffffu, __float_as_uint(f[2 * q + 1] + 8388608.0f) & 1u);
            if (lane == q && w0 + q < W) C[i * ldc + w0 + q] ^= ((uint64_t)hi << 32) | lo;
        }
    }
}

cudaError_t launch_expand_rows(cudaStream_t st, int fmt, const uint64_t *A, int64_t lda, int64_t rows, int64_t k0,
                               int64_t k, int64_t kp, uint8_t *out, int num_sms)
{
    const int64_t total = rows * (kp >> 6);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 16 * num_sms) blocks = 16 * num_sms;
    if (blocks < 1) blocks = 1;
    if (fmt == 4) return launch_kernel(expand_rows_kernel<4>, dim3((int)blocks), dim3(256), 0, st, A, lda, rows, k0, k, kp, out);
    return launch_kernel(expand_rows_kernel<8>, dim3((int)blocks), dim3(256), 0, st, A, lda, rows, k0, k, kp, out);
}

cudaError_t launch_expand_transpose(cudaStream_t st, int fmt, const uint64_t *B, int64_t ldb, int64_t k0, int64_t k,
                                    int64_t n, int64_t kp, uint8_t *out, int num_sms)
{
    const int64_t warps = (kp >> 6) * ((n + 63) >> 6);
    int64_t blocks = (warps * 32 + 255) / 256;
    if (blocks > 16 * num_sms) blocks = 16 * num_sms;
    if (blocks < 1) blocks = 1;
    if (fmt == 4)
        return launch_kernel(expand_transpose_kernel<4>, dim3((int)blocks), dim3(256), 0, st, B, ldb, k0, k, n, kp, out);
    return launch_kernel(expand_transpose_kernel<8>, dim3((int)blocks), dim3(256), 0, st, B, ldb, k0, k, n, kp, out);
}

cudaError_t launch_parity(cudaStream_t st, const float *D, int64_t ldd, int64_t rows, int64_t n, uint64_t *C,
                          int64_t ldc, int num_sms)
{
    const int64_t warps = rows * ((((n + 63) >> 6) + PAR_WORDS - 1) / PAR_WORDS);
    int64_t blocks = (warps * 32 + 255) / 256;
    if (blocks > 16 * num_sms) blocks = 16 * num_sms;
    if (blocks < 1) blocks = 1;
    parity_kernel<<<(int)blocks, 256, 0, st>>>(D, ldd, rows, n, C, ldc);
    return cudaGetLastError();
}

}  // namespace gf2

#ifdef GF2_WITH_CUBLASLT
// ---------------------------------------------------------------------------
// The GEMM: D (rows x n, row-major, ld ldd, fp32) = Ax (rows x kp values,
// K-major) times Bxt^T (Bxt: n x kp values, K-major), by cuBLASLt.  In
// cuBLASLt's column-major terms this is D^T (n x rows) = op(B8t) op(A8) with
// op = transpose for the first operand, both K-major ("TN"); scales are 1.

namespace gf2 {

struct GemmLt {
    cublasLtHandle_t lt = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    uint8_t *ones = nullptr;         // FP4 block scales, all 1.0 (UE4M3 0x38)
    size_t ones_bytes = 0;
};

void *gemm_lt_create()
{
    GemmLt *g = new (std::nothrow) GemmLt();
    if (!g) return nullptr;
    if (cublasLtCreate(&g->lt) != CUBLAS_STATUS_SUCCESS) {
        delete g;
        return nullptr;
    }
    g->ws_bytes = size_t(64) << 20;
    if (cudaMalloc(&g->ws, g->ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        cublasLtDestroy(g->lt);
        delete g;
        return nullptr;
    }
    return g;
}

void gemm_lt_destroy(void *p)
{
    GemmLt *g = static_cast<GemmLt *>(p);
    if (!g) return;
    cudaFree(g->ones);
    cudaFree(g->ws);
    cublasLtDestroy(g->lt);
    delete g;
}

// 0 on success, otherwise a cublasStatus_t value (never 0) or -1 (no memory
// for the scales).  fmt 8: FP8 E4M3 operands of kp bytes a row; fmt 4: FP4
// E2M1 operands of kp / 2 bytes a row, one UE4M3 scale 1.0 per 16 values.
int gemm_counts(void *p, cudaStream_t st, int fmt, const uint8_t *Ax, const uint8_t *Bxt, float *D, int64_t rows,
                int64_t n, int64_t kp, int64_t ldd)
{
    GemmLt *g = static_cast<GemmLt *>(p);
    const cudaDataType_t et = fmt == 4 ? CUDA_R_4F_E2M1 : CUDA_R_8F_E4M3;
    if (fmt == 4) {
        // scale tensors of 128-row x 4-scale tiles: (outer dim rounded up to
        // 128) x (kp / 16) bytes; every entry is 1.0, so A and B share them
        const int64_t outer = ((std::max(rows, n) + 127) / 128) * 128;
        const int64_t inner = ((kp / 16 + 15) / 16) * 16;   // kp / 16 is a multiple of 4; extra room
        const size_t need = (size_t)outer * (size_t)inner + (size_t(1) << 20);
        if (need > g->ones_bytes) {
            cudaFree(g->ones);
            g->ones = nullptr;
            g->ones_bytes = 0;
            if (cudaMalloc(&g->ones, need) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
            g->ones_bytes = need;
            if (cudaMemsetAsync(g->ones, 0x38, need, st) != cudaSuccess) return -1;
        }
    }
    cublasLtMatmulDesc_t op = nullptr;
    cublasLtMatrixLayout_t la = nullptr, lb = nullptr, ld = nullptr;
    cublasLtMatmulPreference_t pref = nullptr;
    cublasStatus_t s = cublasLtMatmulDescCreate(&op, CUBLAS_COMPUTE_32F, CUDA_R_32F);
    const cublasOperation_t ta = CUBLAS_OP_T, tb = CUBLAS_OP_N;
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_TRANSA, &ta, sizeof(ta));
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_TRANSB, &tb, sizeof(tb));
    if (fmt == 4) {
        const int32_t mode = CUBLASLT_MATMUL_MATRIX_SCALE_VEC16_UE4M3;
        const void *sp = g->ones;
        if (s == CUBLAS_STATUS_SUCCESS)
            s = cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_A_SCALE_MODE, &mode, sizeof(mode));
        if (s == CUBLAS_STATUS_SUCCESS)
            s = cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_B_SCALE_MODE, &mode, sizeof(mode));
        if (s == CUBLAS_STATUS_SUCCESS)
            s = cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_A_SCALE_POINTER, &sp, sizeof(sp));
        if (s == CUBLAS_STATUS_SUCCESS)
            s = cublasLtMatmulDescSetAttribute(op, CUBLASLT_MATMUL_DESC_B_SCALE_POINTER, &sp, sizeof(sp));
    }
    // first operand: Bxt, kp x n column-major (ld kp values), transposed -> n x kp
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasLtMatrixLayoutCreate(&la, et, kp, n, kp);
    // second operand: Ax, kp x rows column-major (ld kp values)
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasLtMatrixLayoutCreate(&lb, et, kp, rows, kp);
    // result: n x rows column-major (ld ldd) = rows x n row-major
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasLtMatrixLayoutCreate(&ld, CUDA_R_32F, n, rows, ldd);
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasLtMatmulPreferenceCreate(&pref);
    if (s == CUBLAS_STATUS_SUCCESS)
        s = cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MAX_WORKSPACE_BYTES, &g->ws_bytes,
                                                 sizeof(g->ws_bytes));
    cublasLtMatmulHeuristicResult_t res{};
    int found = 0;
    if (s == CUBLAS_STATUS_SUCCESS) s = cublasLtMatmulAlgoGetHeuristic(g->lt, op, la, lb, ld, ld, pref, 1, &res, &found);
    if (s == CUBLAS_STATUS_SUCCESS && found == 0) s = CUBLAS_STATUS_NOT_SUPPORTED;
    const float alpha = 1.0f, beta = 0.0f;
    if (s == CUBLAS_STATUS_SUCCESS)
        s = cublasLtMatmul(g->lt, op, &alpha, Bxt, la, Ax, lb, &beta, D, ld, D, ld, &res.algo, g->ws, g->ws_bytes, st);
    if (pref) cublasLtMatmulPreferenceDestroy(pref);
    if (ld) cublasLtMatrixLayoutDestroy(ld);
    if (lb) cublasLtMatrixLayoutDestroy(lb);
    if (la) cublasLtMatrixLayoutDestroy(la);
    if (op) cublasLtMatmulDescDestroy(op);
    return s == CUBLAS_STATUS_SUCCESS ? 0 : (int)s;
}

}  // namespace gf2

#else  // library GEMM not built in: the own tcgen05 GEMM (kernels_gemm_f4.cu) is the only one

namespace gf2 {

void *gemm_lt_create() { return nullptr; }
void gemm_lt_destroy(void *) {}
int gemm_counts(void *, cudaStream_t, int, const uint8_t *, const uint8_t *, float *, int64_t, int64_t, int64_t,
                int64_t)
{
    return -1;
}

}  // namespace gf2

#endif
