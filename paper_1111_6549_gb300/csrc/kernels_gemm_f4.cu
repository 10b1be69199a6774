// kernels_gemm_f4.cu -- the GF(2) product C ^= A B as this library's own
// tensor-core GEMM: TMA-fed, warp-specialised tcgen05.mma kind::mxf4 with the
// parity of every count taken out of tensor memory in the epilogue.
//
// Over GF(2), (A B)[i][j] is the parity of the integer count
// sum_k A[i][k] B[k][j] (Section 3.3: Algorithm 3's block step is a matrix
// multiplication; Section 3.2's trailing update A22 += L21 A12 is one).  The
// operands arrive expanded to FP4 E2M1 (1.0 = 0b0010, two per byte, rows of
// A and rows of B^T, both K-major; kernels_gemm.cu's expand kernels), the
// block scales are all 2^0 (UE8M0 0x7F), so the fp32 accumulator holds the
// exact count (below 2^23 by the caller's chunking) and its parity is the
// low mantissa bit of count + 2^23.  No count ever leaves the SM.
//
// Per CTA (persistent, one per SM, 320 threads, 229 KB of shared memory):
//   warp 0    one thread issues the TMA loads: per stage a 256-row x 128-byte
//             box of A and a 192-row x 128-byte box of B^T (256 FP4 values of
//             the inner dimension), 128-byte swizzled, into a 4-stage ring;
//   warp 1    allocates the 512 tensor-memory columns; one thread issues per
//             stage eight MMAs (two M = 128 halves x four K = 64 steps) into
//             two 192-column fp32 accumulators (columns 0 and 256) and
//             commits them to the stage's "empty" barrier;
//   warps 2-9 the epilogue: warp w reads tensor-memory lanes 32 (w % 4) ..
//             of accumulator (w - 2) / 4, 192 counts per row, packs their
//             parities into three words and XORs them into C.
// Tiles of 256 x 192 outputs are walked in groups of eight tile rows so that
// the CTAs running at the same time share their A and B boxes in L2.  Every
// mbarrier wait is bounded (%globaltimer, 2 s); on expiry the kernel records
// GF2_ETIMEOUT, lets its own copies and products in flight finish (bounded),
// frees its tensor memory and returns.
#include "async_dev.cuh"
#include "common.cuh"

#include <cuda.h>

#include <algorithm>

namespace gf2 {

namespace {

constexpr int G_BM = 256;                                   // tile rows (two M = 128 halves)
constexpr int G_BN = 192;                                   // tile columns (three words)
constexpr int G_KB = 128;                                   // bytes of one row per stage (256 values)
constexpr int G_STAGES = 4;
constexpr int G_A_BYTES = G_BM * G_KB;                      // 32 KiB
constexpr int G_B_BYTES = G_BN * G_KB;                      // 24 KiB
constexpr int G_STAGE_BYTES = G_A_BYTES + G_B_BYTES;        // 56 KiB
constexpr int G_THREADS = 320;
constexpr int G_EPI_WARPS = 8;
constexpr uint32_t G_TMEM_COLS = 512;
constexpr uint32_t G_ACC1 = 256;                            // second accumulator's first column
constexpr uint32_t G_SF = 448;                              // 64 columns of block scales
constexpr int G_GROUP = 8;                                  // tile rows per scheduling group
constexpr size_t G_SMEM = (size_t)G_STAGES * G_STAGE_BYTES + 1024 + 256;
static_assert(G_SMEM <= 232448, "gemm_f4 shared memory");
// kind::mxf4 instruction descriptor: A and B E2M1 (1 at bits 7-9, 10-12),
// K-major, N >> 3 at bit 17, UE8M0 scales (bit 23), M >> 4 at bit 24
// (M = 128), scale-factor IDs 0, K = 64.
constexpr uint32_t G_IDESC = (1u << 7) | (1u << 10) | ((uint32_t)(G_BN >> 3) << 17) | (1u << 23) |
                             ((128u >> 4) << 24);

// shared-memory descriptor of a K-major operand in the 128-byte swizzled
// layout TMA writes: rows 128 bytes apart, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t g_desc_sw128(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                                 // leading offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;                       // 8-row group stride
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;                                 // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void g_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t sf, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %5, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%4], p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(G_IDESC), "r"(sf), "r"(acc));
}

__device__ __forceinline__ void g_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void g_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void g_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void g_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void g_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// 32 parities of 32 fp32 counts (count + 2^23 keeps the integer in the low
// mantissa bits)
__device__ __forceinline__ uint32_t g_parity32(const uint32_t (&v)[32])
{
    uint32_t p = 0;
#pragma unroll
    for (int q = 0; q < 32; ++q) p |= (__float_as_uint(__uint_as_float(v[q]) + 8388608.0f) & 1u) << q;
    return p;
}

struct GemmF4Args {
    uint64_t *C;
    int64_t ldc;
    int64_t m, n;          // output rows (valid rows of A) and columns
    int64_t kstages;       // stages of 256 inner values
    int32_t *err;
};

// tile t -> (tile row, tile column), groups of G_GROUP tile rows walked column by column
__device__ __forceinline__ void g_tile(int64_t t, int64_t TM, int64_t TN, int64_t &tm, int64_t &tn)
{
    const int64_t per = (int64_t)G_GROUP * TN;
    const int64_t grp = t / per, in = t - grp * per;
    const int64_t rows = min((int64_t)G_GROUP, TM - grp * G_GROUP);
    tm = grp * G_GROUP + in % rows;
    tn = in / rows;
}

}  // namespace

__global__ void __launch_bounds__(G_THREADS, 1)
    gemm_f4_kernel(const __grid_constant__ TensorMap2D tmA, const __grid_constant__ TensorMap2D tmB, GemmF4Args a)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(1024) uint8_t g_smem[];
    uint8_t *stages = g_smem + ((1024u - (smem_u32(g_smem) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(stages + G_STAGES * G_STAGE_BYTES);
    uint64_t *empty = full + G_STAGES;
    uint64_t *tfull = empty + G_STAGES;
    uint64_t *tempty = tfull + 1;
    uint64_t *done = tempty + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t TM = (a.m + G_BM - 1) / G_BM, TN = (a.n + G_BN - 1) / G_BN;
    const int64_t T = TM * TN;

    if (tid == 0) {
        for (int s = 0; s < G_STAGES; ++s) {
            mbar_init_cta(&full[s], 1);
            mbar_init_cta(&empty[s], 1);
        }
        mbar_init_cta(tfull, 1);
        mbar_init_cta(tempty, G_EPI_WARPS);
        mbar_init_cta(done, 1);
        *abort_flag = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(G_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    mbar_init_fence();
    g_fence_before();
    __syncthreads();
    g_fence_after();
    const uint32_t tmem = *tmem_slot;
    // block scales 2^0 in every byte of the 64 columns from G_SF, all 128
    // lanes (warps 2..5 cover the four lane quarters)
    if (warp >= 2 && warp < 6) {
        const uint32_t x = 0x7F7F7F7Fu;
#pragma unroll
        for (int c = 0; c < 2; ++c)
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
                "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(
                    tmem + ((uint32_t)(32 * (warp & 3)) << 16) + G_SF + 32 * c),
                "r"(x)
                : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    }
    g_fence_before();
    __syncthreads();
    g_fence_after();

    auto fail = [&]() {
        *abort_flag = 1;
        if (a.err) atomicExch(a.err, 4);                     // GF2_ETIMEOUT
    };

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int64_t it = 0;
            for (int64_t t = blockIdx.x; t < T && !*abort_flag; t += gridDim.x) {
                int64_t tm, tn;
                g_tile(t, TM, TN, tm, tn);
                for (int64_t ks = 0; ks < a.kstages; ++ks, ++it) {
                    const int s = (int)(it % G_STAGES);
                    const uint32_t use = (uint32_t)(it / G_STAGES);
                    if (!mbar_wait_limited(&empty[s], (use & 1u) ^ 1u)) { fail(); break; }
                    if (*abort_flag) break;
                    uint8_t *sa = stages + s * G_STAGE_BYTES;
                    mbar_expect_tx(&full[s], G_STAGE_BYTES);
                    tma_load_2d(sa, &tmA, (int)(ks * G_KB), (int)(tm * G_BM), &full[s]);
                    tma_load_2d(sa + G_A_BYTES, &tmB, (int)(ks * G_KB), (int)(tn * G_BN), &full[s]);
                }
            }
            // copies still in flight land before the CTA can exit
            for (int64_t j = it - 1; j >= 0 && j >= it - G_STAGES; --j)
                mbar_wait_limited(&full[j % G_STAGES], (uint32_t)((j / G_STAGES) & 1));
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int64_t it = 0, tc = 0;
            for (int64_t t = blockIdx.x; t < T && !*abort_flag; t += gridDim.x, ++tc) {
                if (!mbar_wait_limited(tempty, ((uint32_t)tc & 1u) ^ 1u)) { fail(); break; }
                g_fence_after();
                for (int64_t ks = 0; ks < a.kstages; ++ks, ++it) {
                    const int s = (int)(it % G_STAGES);
                    if (!mbar_wait_limited(&full[s], (uint32_t)((it / G_STAGES) & 1))) { fail(); break; }
                    g_fence_after();
                    const uint32_t sa = smem_u32(stages + s * G_STAGE_BYTES);
                    const uint32_t sb = sa + G_A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t acc = (ks > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t bd = g_desc_sw128(sb + 32 * kk);
                        g_mma(tmem, g_desc_sw128(sa + 32 * kk), bd, tmem + G_SF, acc);
                        g_mma(tmem + G_ACC1, g_desc_sw128(sa + 128 * G_KB + 32 * kk), bd, tmem + G_SF, acc);
                    }
                    g_commit(&empty[s]);
                }
                if (*abort_flag) break;
                g_commit(tfull);
            }
            // every product issued has completed before tensor memory is released
            g_commit(done);
            if (!mbar_wait_limited(done, 0)) fail();
        }
    } else {
        // ---------------- epilogue
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int64_t Wc = (a.n + 63) >> 6;
        int64_t tc = 0;
        for (int64_t t = blockIdx.x; t < T; t += gridDim.x, ++tc) {
            if (*abort_flag) break;
            if (!mbar_wait_limited(tfull, (uint32_t)tc & 1u)) { fail(); break; }
            g_fence_after();
            int64_t tm, tn;
            g_tile(t, TM, TN, tm, tn);
            uint64_t words[3];
            const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)h * G_ACC1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint32_t v[32];
                g_ld32(base + 64 * c, v);
                const uint32_t lo = g_parity32(v);
                g_ld32(base + 64 * c + 32, v);
                const uint32_t hi = g_parity32(v);
                words[c] = ((uint64_t)hi << 32) | lo;
            }
            g_fence_before();
            __syncwarp();
            if (lane == 0) g_arrive(tempty);                 // accumulators free for the next tile
            const int64_t i = tm * G_BM + 128 * h + 32 * q + lane;
            if (i < a.m) {
                uint64_t *row = a.C + i * a.ldc;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int64_t w = 3 * tn + c;
                    if (w < Wc && words[c]) row[w] ^= words[c];
                }
            }
        }
    }
    g_fence_before();
    __syncthreads();
    g_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(G_TMEM_COLS));
}

// Encode the TMA descriptor of `rows` rows of `rowb` bytes (the expanded
// operand), boxes of `box_rows` rows x 128 bytes, 128-byte swizzle.
bool encode_f4_operand(TensorMap2D *out, const uint8_t *base, int64_t rows, int64_t rowb, int box_rows);

cudaError_t launch_gemm_f4(cudaStream_t st, uint64_t *C, int64_t ldc, const uint8_t *A4, int64_t a_rows,
                           const uint8_t *B4t, int64_t b_rows, int64_t m, int64_t n, int64_t kp, int32_t *err,
                           int num_sms)
{
    if (m <= 0 || n <= 0 || kp <= 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(gemm_f4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t rowb = kp / 2;
    TensorMap2D ta{}, tb{};
    if (a_rows < m || b_rows < n || !encode_f4_operand(&ta, A4, a_rows, rowb, G_BM) ||
        !encode_f4_operand(&tb, B4t, b_rows, rowb, G_BN))
        return cudaErrorInvalidValue;
    GemmF4Args a{C, ldc, m, n, (rowb + G_KB - 1) / G_KB, err};
    const int64_t tiles = ((m + G_BM - 1) / G_BM) * ((n + G_BN - 1) / G_BN);
    const int grid = (int)std::min<int64_t>(num_sms, std::max<int64_t>(tiles, 1));
    return launch_kernel(gemm_f4_kernel, dim3(grid), dim3(G_THREADS), G_SMEM, st, ta, tb, a);
}

}  // namespace gf2
