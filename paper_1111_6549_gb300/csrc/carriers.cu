// carriers.cu -- measured rates of the tensor-core forms that can carry a
// GF(2) product, and an exactness check of each.
//
// A GF(2) product C = A B is an integer product reduced mod 2 (Section 3.3:
// the block step of Algorithm 3 is a matrix multiplication; Section 3.2's
// trailing update A22 += L21 A12 is one with inner dimension k).  On the
// tensor cores the 0/1 operands can be carried as
//   b1    mma.sync m16n8k256 .b1 AND + POPC (int32 counts), the legacy warp
//         path;
//   fp8   tcgen05.mma kind::f8f6f4, E4M3 1.0 = 0x38, fp32 counts;
//   fp4   tcgen05.mma kind::mxf4 with block scales (UE8M0, all 2^0, one per
//         32 elements), E2M1 1.0 = 0x2 packed two per byte, fp32 counts;
//   nvf4  tcgen05.mma kind::mxf4nvf4, the same E2M1 operands with UE4M3
//         scales (all 1.0 = 0x38) one per 16 elements (scale_vec::4X).
// (kind::i8 is not accepted for sm_103a by this toolkit's assembler.)
// gf2_carrier_rate() runs one kernel of each carrier on every SM with the
// operands resident (registers or shared memory) and reports multiply-adds
// per second; gf2_carrier_check() multiplies a 128 x 64 by a 64 x 256 bit
// matrix with one instruction sequence of the carrier and returns the counts.
// Every wait for a tensor-core commit is bounded (%globaltimer).
#include "common.cuh"
#include "gf2.h"

#include <algorithm>

namespace gf2 {

namespace {

constexpr int CR_THREADS = 128;
constexpr uint32_t CR_TMEM_COLS = 512;          // 256 accumulator columns + scale columns at 256
constexpr uint32_t CR_SCALE_COL = 256;
constexpr unsigned long long CR_WAIT_NS = 2000000000ull;
constexpr int CR_PAD_SMEM = 160 * 1024;         // rate runs: unused, keeps one CTA (one TMEM user) per SM

// kind::f8f6f4: D f32 (bits 4-5 = 1), A and B E4M3 (0), K-major, N >> 3 at
// bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC_F8 = (1u << 4) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
// kind::mxf4 block-scaled: scale-factor IDs 0 (bits 4-5, 29-30), A and B
// E2M1 (1 at bits 7-9 and 10-12), K-major, N >> 3 at bit 17, scale type
// UE8M0 (bit 23), M >> 4 at bit 24 (M = 128), K = 64.
constexpr uint32_t IDESC_F4 = (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | (1u << 23) | ((128u >> 4) << 24);
// kind::mxf4nvf4 with scale_vec::4X: as above with scale type UE4M3 (bit 23 = 0).
constexpr uint32_t IDESC_NVF4 = (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t cr_saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long cr_now()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool cr_wait(uint64_t *bar, uint32_t phase)
{
    const unsigned long long t0 = cr_now();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(cr_saddr(bar)), "r"(phase)
            : "memory");
        if (ok) return true;
        if (cr_now() - t0 > CR_WAIT_NS) return false;
    }
}

__device__ __forceinline__ uint64_t cr_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void cr_mma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC_F8), "r"(acc));
}

__device__ __forceinline__ void cr_mma_f4(uint32_t d, uint64_t a, uint64_t b, uint32_t sfa, uint32_t sfb,
                                          uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC_F4), "r"(sfa), "r"(sfb), "r"(acc));
}

__device__ __forceinline__ void cr_mma_nvf4(uint32_t d, uint64_t a, uint64_t b, uint32_t sfa, uint32_t sfb,
                                            uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4nvf4.block_scale.scale_vec::4X [%0], %1, %2, %3, [%4], [%5], p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC_NVF4), "r"(sfa), "r"(sfb), "r"(acc));
}

__device__ __forceinline__ void cr_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(cr_saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void cr_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void cr_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 32 lanes x 32 columns of tensor memory -> 32 registers per thread
__device__ __forceinline__ void cr_ld32(uint32_t taddr, uint32_t (&v)[32])
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

// one value in 32 columns of this warp's 32 lanes
__device__ __forceinline__ void cr_st32(uint32_t taddr, uint32_t x)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(taddr),
        "r"(x)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// Byte offset of (row, 16-byte K group j) in the no-swizzle K-major
// core-matrix layout with G groups per row: K-direction stride 128 bytes,
// 8-row groups G * 128 bytes apart.
__device__ __forceinline__ uint32_t cr_core(int row, int j, int G)
{
    return (uint32_t)(((row >> 3) * G + j) * 128 + (row & 7) * 16);
}

// 64 operand bits of one row -> the carrier's encoding in shared memory
__device__ __forceinline__ void cr_expand(uint8_t *tile, int row, uint64_t bits, int carrier)
{
    if (carrier == GF2_CARRIER_FP8) {
        for (int j = 0; j < 4; ++j) {                  // 16 elements per 16-byte group
            uint8_t v[16];
            for (int e = 0; e < 16; ++e) v[e] = ((bits >> (16 * j + e)) & 1ull) ? 0x38 : 0x00;
            for (int e = 0; e < 16; ++e) tile[cr_core(row, j, 4) + e] = v[e];
        }
    } else {
        for (int j = 0; j < 2; ++j) {                  // 32 elements per 16-byte group
            for (int e = 0; e < 16; ++e) {
                const int k = 32 * j + 2 * e;
                const uint8_t lo = ((bits >> k) & 1ull) ? 0x2 : 0x0;
                const uint8_t hi = ((bits >> (k + 1)) & 1ull) ? 0x2 : 0x0;
                tile[cr_core(row, j, 2) + e] = (uint8_t)(lo | (hi << 4));
            }
        }
    }
}

struct CrArgs {
    int carrier;
    int64_t iters;
    const uint64_t *a;   // check: 128 rows of 64 bits
    const uint64_t *b;   // check: 256 columns of 64 bits (B transposed)
    int32_t *counts;     // check: 128 x 256; rate: one count per CTA
    int32_t *err;
};

// Tensor-core carriers: one CTA of 128 threads per SM.  Check mode (iters <
// 0): one product of the given bits.  Rate mode: iters instructions issued
// back to back into one accumulator on all-ones operands (each adds K).
__global__ void __launch_bounds__(CR_THREADS, 1) carrier_tc_kernel(CrArgs a)
{
    __shared__ __align__(1024) uint8_t sA[128 * 64];
    __shared__ __align__(1024) uint8_t sB[256 * 64];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool check = a.iters < 0;
    const int carrier = a.carrier;

    for (int row = tid; row < 128; row += CR_THREADS) cr_expand(sA, row, check ? a.a[row] : ~0ull, carrier);
    for (int row = tid; row < 256; row += CR_THREADS) cr_expand(sB, row, check ? a.b[row] : ~0ull, carrier);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(cr_saddr(&bar)) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(cr_saddr(&tmem_base)),
                     "r"(CR_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    cr_fence_before();
    __syncthreads();
    cr_fence_after();
    const uint32_t tmem = tmem_base;
    // block scales 1.0 in every byte of 32 columns, all lanes: UE8M0 0x7F, UE4M3 0x38
    if (carrier == GF2_CARRIER_FP4) cr_st32(tmem + ((uint32_t)(32 * warp) << 16) + CR_SCALE_COL, 0x7F7F7F7Fu);
    if (carrier == GF2_CARRIER_NVF4) cr_st32(tmem + ((uint32_t)(32 * warp) << 16) + CR_SCALE_COL, 0x38383838u);
    cr_fence_before();
    __syncthreads();
    cr_fence_after();

    bool ok = true;
    if (tid == 0) {
        const uint32_t a0 = cr_saddr(sA), b0 = cr_saddr(sB);
        const uint32_t sf = tmem + CR_SCALE_COL;
        const int64_t n = check ? 1 : a.iters;
        for (int64_t i = 0; i < n; ++i) {
            if (carrier == GF2_CARRIER_FP8) {
                // two K = 32 steps over the 64-byte rows (4 groups per row)
                cr_mma_f8(tmem, cr_desc(a0, 128, 512), cr_desc(b0, 128, 512), i > 0 ? 1u : 0u);
                cr_mma_f8(tmem, cr_desc(a0 + 256, 128, 512), cr_desc(b0 + 256, 128, 512), 1u);
            } else if (carrier == GF2_CARRIER_FP4) {
                // one K = 64 step over the 32-byte rows (2 groups per row)
                cr_mma_f4(tmem, cr_desc(a0, 128, 256), cr_desc(b0, 128, 256), sf, sf, i > 0 ? 1u : 0u);
            } else {
                cr_mma_nvf4(tmem, cr_desc(a0, 128, 256), cr_desc(b0, 128, 256), sf, sf, i > 0 ? 1u : 0u);
            }
        }
        cr_commit(&bar);
    }
    __syncwarp();
    if (!cr_wait(&bar, 0)) {
        ok = false;
        if (a.err) atomicExch(a.err, GF2_ETIMEOUT);
    }
    cr_fence_after();
    if (ok) {
        // warp w reads lanes 32w .. 32w + 31 (rows), 32 columns at a time
        const int row = 32 * warp + (tid & 31);
        const int ncol = check ? 256 : 32;
        for (int c0 = 0; c0 < ncol; c0 += 32) {
            uint32_t v[32];
            cr_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            if (check) {
                for (int q = 0; q < 32; ++q) a.counts[row * 256 + c0 + q] = (int32_t)__uint_as_float(v[q]);
            } else if (row == 0 && c0 == 0) {
                a.counts[blockIdx.x] = (int32_t)__uint_as_float(v[0]);
            }
        }
    }
    cr_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(CR_TMEM_COLS));
}

// The b1 warp-level carrier: m16n8k256, AND + POPC into int32.  Check mode:
// A rows from a.a (16 rows x 256 bits as four words each), B columns from
// a.b (8 columns x 4 words); rate mode: four independent accumulator sets
// per warp on all-ones registers.
__global__ void __launch_bounds__(256) carrier_b1_kernel(CrArgs a)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    if (a.iters < 0) {
        if (blockIdx.x != 0 || threadIdx.x >= 32) return;
        // fragment layout of m16n8k256 .b1 (row-major A, column-major B):
        // a0: row g, bits 32t .. 32t+31; a1: row g+8, same bits; a2, a3: bits 128 + 32t ..
        // b0: column g, bits 32t ..; b1: column g, bits 128 + 32t ..
        const uint32_t *A32 = reinterpret_cast<const uint32_t *>(a.a);
        const uint32_t *B32 = reinterpret_cast<const uint32_t *>(a.b);
        const uint32_t a0 = A32[g * 8 + t], a1 = A32[(g + 8) * 8 + t];
        const uint32_t a2 = A32[g * 8 + 4 + t], a3 = A32[(g + 8) * 8 + 4 + t];
        const uint32_t b0 = B32[g * 8 + t], b1 = B32[g * 8 + 4 + t];
        int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        asm volatile(
            "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+r"(c0), "+r"(c1), "+r"(c2), "+r"(c3)
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        // c0, c1: row g, columns 2t, 2t+1; c2, c3: row g + 8
        a.counts[g * 8 + 2 * t] = c0;
        a.counts[g * 8 + 2 * t + 1] = c1;
        a.counts[(g + 8) * 8 + 2 * t] = c2;
        a.counts[(g + 8) * 8 + 2 * t + 1] = c3;
        return;
    }
    const uint32_t x = ~0u;
    int c[4][4] = {};
    for (int64_t i = 0; i < a.iters; ++i) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
            asm volatile(
                "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+r"(c[s][0]), "+r"(c[s][1]), "+r"(c[s][2]), "+r"(c[s][3])
                : "r"(x), "r"(x), "r"(x), "r"(x), "r"(x), "r"(x));
    }
    // one count per CTA for the exactness check; the other chains feed a
    // value the compiler cannot drop
    if (threadIdx.x == 0) a.counts[blockIdx.x] = c[0][0];
    if (c[1][1] + c[2][2] + c[3][3] == 1) a.counts[blockIdx.x] = -1;
}

}  // namespace

}  // namespace gf2

using namespace gf2;

extern "C" {

int gf2_carrier_check(int carrier, const uint64_t *a_bits, const uint64_t *b_bits, int32_t *counts)
{
    if (!a_bits || !b_bits || !counts) return GF2_EINVAL;
    if (carrier != GF2_CARRIER_B1 && carrier != GF2_CARRIER_FP8 && carrier != GF2_CARRIER_FP4 &&
        carrier != GF2_CARRIER_NVF4)
        return GF2_EINVAL;
    int32_t *err = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&err), sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return GF2_ENOMEM;
    }
    cudaMemset(err, 0, sizeof(int32_t));
    CrArgs args{carrier, -1, a_bits, b_bits, counts, err};
    if (carrier == GF2_CARRIER_B1) carrier_b1_kernel<<<1, 32>>>(args);
    else carrier_tc_kernel<<<1, CR_THREADS>>>(args);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int32_t herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) { cudaGetLastError(); return GF2_ECUDA; }
    return herr ? herr : GF2_OK;
}

int gf2_carrier_rate(int carrier, int64_t iters, double *macs_per_s, int64_t *count_out)
{
    if (!macs_per_s || iters <= 0) return GF2_EINVAL;
    if (carrier != GF2_CARRIER_B1 && carrier != GF2_CARRIER_FP8 && carrier != GF2_CARRIER_FP4 &&
        carrier != GF2_CARRIER_NVF4)
        return GF2_EINVAL;
    // exact counts: every accumulator stays below 2^24 (fp32) / 2^31 (int32)
    const int64_t per = carrier == GF2_CARRIER_B1 ? 256 : 64;
    if (iters * per >= (carrier == GF2_CARRIER_B1 ? (int64_t(1) << 31) : (int64_t(1) << 24))) return GF2_EINVAL;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = carrier == GF2_CARRIER_B1 ? 4 * sms : sms;
    int32_t *buf = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&buf), (size_t)(grid + 1) * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return GF2_ENOMEM;
    }
    cudaMemset(buf, 0, (size_t)(grid + 1) * sizeof(int32_t));
    CrArgs args{carrier, iters, nullptr, nullptr, buf, buf + grid};
    if (carrier != GF2_CARRIER_B1 &&
        cudaFuncSetAttribute(carrier_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CR_PAD_SMEM) !=
            cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        return GF2_ECUDA;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        if (carrier == GF2_CARRIER_B1) carrier_b1_kernel<<<grid, 256>>>(args);
        else carrier_tc_kernel<<<grid, CR_THREADS, CR_PAD_SMEM>>>(args);
    };
    launch();                                         // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int32_t host[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(&host[0], buf, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&host[1], buf + grid, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) { cudaGetLastError(); return GF2_ECUDA; }
    if (host[1]) return host[1];
    // multiply-adds per launch: b1 16 x 8 x 256 per instruction, four chains
    // per warp, eight warps per CTA; tcgen05 128 x 256 x 64 per issue step
    const double per_iter = carrier == GF2_CARRIER_B1 ? 4.0 * 8.0 * 16 * 8 * 256 : 128.0 * 256 * 64;
    *macs_per_s = (double)grid * (double)iters * per_iter / (ms * 1e-3);
    if (count_out) *count_out = host[0];
    return GF2_OK;
}

}  // extern "C"
