// kernels_tc.cu -- the trailing update / product on the 5th-generation tensor
// cores (tcgen05), exact over GF(2).
//
// For a tile of 128 rows x 256 columns: D = X * G^T counts, over GF(2)
// generators G (K rows of 256 column bits) and per-row coefficient words X
// (K bits per row), and the row's bits flip where the count is odd:
//     row[col] ^= parity( sum_k X[row][k] * G[k][col] ).
// This is the same update as the tabulated one (Section 3.2's A22 += L21 A12,
// or C ^= A B), computed as an integer matrix product and reduced mod 2, which
// is exact because every operand is 0 or 1 and every count stays below 2^23.
//
//  * operands: 0/1 as FP8 E4M3 (1.0 = 0x38), both K-major, in the canonical
//    no-swizzle layout of 8-row x 16-byte core matrices (K-direction stride
//    128 bytes, row-direction stride 512 bytes for a 64-byte K chunk);
//  * one elected thread issues tcgen05.mma (kind::f8f6f4, M = 128, N = 256,
//    K = 32 per instruction) into a 256-column fp32 accumulator in tensor
//    memory, and tcgen05.commit signals an mbarrier;
//  * the epilogue reads the counts with tcgen05.ld (32 lanes x 32 columns per
//    warp and instruction), takes the parity by adding 2^23 (the integer then
//    sits in the low mantissa bits) and packs 64 parities per word.
// Every mbarrier wait is bounded; on expiry the kernel records GF2_ETIMEOUT in
// the error word, frees its tensor memory and returns.
#include "common.cuh"

#include <algorithm>

namespace gf2 {

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;
constexpr int TC_N = 256;
constexpr int TC_KC = 64;                                   // K chunk: 64 generators
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr uint32_t TC_IDESC = (1u << 4)                     // D: f32
                              | (0u << 7) | (0u << 10)      // A, B: E4M3
                              | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
constexpr int TC_A_BYTES = TC_M * TC_KC;                    // 8 KiB
constexpr int TC_B_BYTES = TC_N * TC_KC;                    // 16 KiB
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // 2 s: far beyond any product here

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase, giving up after TC_WAIT_NS.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase)
{
    const unsigned long long t0 = gtime();
    while (!mbar_try_wait(bar, phase))
        if (gtime() - t0 > TC_WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Shared-memory matrix descriptor: start, K-direction and row-direction core
// matrix strides (bytes), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
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

__device__ __forceinline__ unsigned transpose32_tc(unsigned x)
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

// Byte offset of (row, 16-byte K group j) in the core-matrix layout of a
// 64-byte-per-row K chunk.
__device__ __forceinline__ uint32_t core_off(int row, int j) { return (uint32_t)(((row >> 3) * 4 + j) * 128 + (row & 7) * 16); }

// 64 bits -> 64 E4M3 bytes (1.0 where the bit is set), as four 16-byte groups.
__device__ __forceinline__ void expand_store(uint8_t *tile, int row, uint64_t bits, const uint64_t *lut)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint64_t lo = lut[(bits >> (16 * j)) & 255u];
        const uint64_t hi = lut[(bits >> (16 * j + 8)) & 255u];
        *reinterpret_cast<ulonglong2 *>(tile + core_off(row, j)) = make_ulonglong2(lo, hi);
    }
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS, 1) tc_update_kernel(UpdArgs a)
{
    __shared__ __align__(1024) uint8_t sA[TC_A_BYTES];
    __shared__ __align__(1024) uint8_t sB[TC_B_BYTES];
    __shared__ uint64_t lut[256];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ const uint64_t *sGen[KS];
    __shared__ int s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const StripeDesc *d = a.desc;
    int64_t row_lo, row_hi, w_lo, r = 0;
    int maxpos = -1, nS = 0, nchunks = 1;
    const int64_t W = a.W;
    if (a.mode == UPD_PLE) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        r = d->r;
        row_lo = r;
        row_hi = a.m;
        w_lo = (d->c >> 6) + (a.first_off > 0 ? a.first_off : 1);
        maxpos = d->maxpos;
        nS = d->nS;
        if (tid < KS) sGen[tid] = (tid < rbar) ? a.S + tid * a.ldS : nullptr;
    } else if (a.mode == UPD_RREF) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        row_lo = a.row_lo;                    // 0, or the first row of a block's own RREF
        row_hi = d->r;
        w_lo = max((int64_t)(d->c >> 6), a.w_lo);  // a.w_lo > 0: only a right part of the row
        if (tid < KS) sGen[tid] = nullptr;
        __syncthreads();
        if (tid < rbar) sGen[d->qbar[tid]] = a.A + (d->r + tid) * a.ld;
    } else {
        row_lo = a.row_lo;
        row_hi = a.row_hi;
        w_lo = a.w_lo;
        nchunks = (int)((a.gen_count + TC_KC - 1) / TC_KC);
    }
    // E4M3 expansion of a byte: 0x38 (1.0) in every byte whose bit is set
    for (int b = tid; b < 256; b += TC_THREADS) {
        uint64_t v = 0;
        for (int i = 0; i < 8; ++i)
            if ((b >> i) & 1) v |= 0x38ull << (8 * i);
        lut[b] = v;
    }
    if (tid == 0) { mbar_init(&mbar, 1); s_abort = 0; }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(&tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    // PLE: staged rows get their left part (old L bits, new L bits, stripe)
    if (a.mode == UPD_PLE && a.left_copies) {
        for (int k = blockIdx.x; k < nS; k += gridDim.x) {
            const uint64_t *src = a.S + (int64_t)k * a.ldS;
            uint64_t *dst = a.A + (r + d->S_off[k]) * a.ld;
            for (int64_t w = tid; w < w_lo; w += TC_THREADS) dst[w] = src[w];
        }
    }

    const int64_t R = row_hi - row_lo;
    uint32_t phase = 0;
    if (R > 0 && w_lo < W) {
        const int64_t x0 = w_lo / 4, x1 = (W + 3) / 4;     // 256-column tiles, word aligned
        const int64_t NTX = x1 - x0, NTY = (R + TC_M - 1) / TC_M;
        const int64_t T = NTX * NTY;
        const int64_t t_beg = T * blockIdx.x / gridDim.x, t_end = T * (blockIdx.x + 1) / gridDim.x;
        if (blockIdx.x == 0 && tid == 0 && a.bytes)
            atomicAdd(a.bytes, (unsigned long long)(R * (W - w_lo) * 16));
        int64_t b_tile = -1;                               // tile whose generators sit in sB
        for (int64_t t = t_beg; t < t_end; ++t) {
            const int64_t tx = x0 + t / NTY, ty = t % NTY;
            const int64_t wb = tx * 4;
            const int64_t row0 = row_lo + ty * TC_M;
            for (int kc = 0; kc < nchunks; ++kc) {
                // ---- operands: coefficient rows -> sA, generators -> sB
                {
                    const int64_t i = row0 + tid;
                    uint64_t x = 0;
                    if (i < row_hi) x = (a.mode == UPD_MUL) ? a.idx[i * a.idx_stride + kc] : a.idx[i * a.idx_stride];
                    if (a.mode == UPD_MUL) {
                        const int64_t rem = a.gen_count - (int64_t)kc * TC_KC;
                        if (rem < 64) x &= (rem <= 0) ? 0ull : ((1ull << rem) - 1ull);
                    }
                    expand_store(sA, tid, x, lut);
                }
                if (a.mode == UPD_MUL || b_tile != tx) {
                    // warp w transposes generator word wb + w (64 columns) over 64 generators
                    const int64_t word = wb + warp;
                    uint64_t g0 = 0, g1 = 0;
                    if (word < W) {
                        if (a.mode == UPD_MUL) {
                            const int64_t k0 = (int64_t)kc * TC_KC;
                            if (k0 + lane < a.gen_count) g0 = a.B[(k0 + lane) * a.ldb + word];
                            if (k0 + 32 + lane < a.gen_count) g1 = a.B[(k0 + 32 + lane) * a.ldb + word];
                        } else {
                            const uint64_t *p0 = sGen[lane], *p1 = sGen[32 + lane];
                            if (p0) g0 = p0[word];
                            if (p1) g1 = p1[word];
                        }
                    }
                    const unsigned c0a = transpose32_tc((unsigned)g0), c1a = transpose32_tc((unsigned)(g0 >> 32));
                    const unsigned c0b = transpose32_tc((unsigned)g1), c1b = transpose32_tc((unsigned)(g1 >> 32));
                    // lane c: column 64w + c and 64w + 32 + c, 64 generator bits each
                    expand_store(sB, warp * 64 + lane, ((uint64_t)c0b << 32) | c0a, lut);
                    expand_store(sB, warp * 64 + 32 + lane, ((uint64_t)c1b << 32) | c1a, lut);
                    b_tile = tx;
                }
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const uint32_t a0 = saddr(sA), b0 = saddr(sB);
#pragma unroll
                    for (int ks = 0; ks < TC_KC / 32; ++ks)
                        mma_f8(tmem, smem_desc(a0 + ks * 256, 128, 512), smem_desc(b0 + ks * 256, 128, 512),
                               (kc > 0 || ks > 0) ? 1u : 0u);
                    mma_commit(&mbar);
                }
                // all threads wait for the products (the operand buffers are reused next)
                if (!mbar_wait_bounded(&mbar, phase)) {
                    s_abort = 1;
                    if (a.err) atomicExch(a.err, 4);   // GF2_ETIMEOUT
                }
                __syncthreads();                             // one decision for the whole block
                if (s_abort) break;
                phase ^= 1u;
                tc_fence_after();
            }
            if (s_abort) break;
            // ---- epilogue: parity of the counts, XOR into the rows
            const int64_t i = row0 + warp * 32 + lane;
            const uint64_t *src = nullptr;
            uint64_t *dst = nullptr;
            if (i < row_hi) {
                src = a.A + i * a.ld;
                if (a.mode == UPD_PLE && i - r <= maxpos) {
                    const int mv = a.map[i];
                    if (mv >= 0 && (mv >> 8) == a.stripe) src = a.S + (int64_t)(mv & 255) * a.ldS;
                }
                dst = a.A + i * a.ld;
            }
#pragma unroll 1
            for (int cb = 0; cb < 8; cb += 2) {
                uint32_t v0[32], v1[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), v0);
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((cb + 1) * 32), v1);
                uint32_t p0 = 0, p1 = 0;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    p0 |= (__float_as_uint(__uint_as_float(v0[q]) + 8388608.0f) & 1u) << q;
                    p1 |= (__float_as_uint(__uint_as_float(v1[q]) + 8388608.0f) & 1u) << q;
                }
                const int64_t w = wb + cb / 2;
                if (dst && w >= w_lo && w < W) dst[w] = src[w] ^ (((uint64_t)p1 << 32) | p0);
            }
            tc_fence_before();
            __syncthreads();                                 // TMEM and sA free for the next tile
            tc_fence_after();
        }
    }
    if (s_abort) {
        // the last product may still be running: wait for it (bounded) before
        // its tensor memory is released
        mbar_wait_bounded(&mbar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ---------------------------------------------------------------------------
// The product C ^= A B (A: m x k bits, B: k x n bits) as a pipelined tcgen05
// kernel.  Per CTA output tile of 256 rows x 256 columns, two M = 128
// accumulators (all 512 tensor-memory columns) share each expanded chunk of
// B; per chunk of 128 inner-dimension bits all 512 threads expand their
// operand bits to FP8 (arithmetic nibble spread, no table lookups) into one
// of two shared-memory stages while the MMAs of the previous chunk run from
// the other stage; one thread issues the eight MMAs of a chunk and commits
// them to that stage's mbarrier, which frees the stage again.  The operand
// bits come through a shared-memory ring filled by cp.async five chunks
// ahead (a load that ends in a register would stall the chunk on memory
// latency).  The epilogue takes
// each count's parity (count + 2^23) and XORs 64 of them per word into C.
constexpr int TM_THREADS = 512;
constexpr int TM_KW = 2;                                     // inner-dimension words per chunk (128 bits)
constexpr int TM_KB = 64 * TM_KW;                            // FP8 bytes per operand row and chunk
constexpr int TM_A_BYTES = TC_M * TM_KB;                     // 16 KiB: 128 rows x 128 bytes
constexpr int TM_B_BYTES = TC_N * TM_KB;                     // 32 KiB: 256 columns x 128 bytes
constexpr int TM_STAGE_BYTES = 2 * TM_A_BYTES + TM_B_BYTES;  // 64 KiB
constexpr uint32_t TM_TMEM_COLS = 512;
constexpr int TM_RING = 6;                                   // chunks of operand bits in flight
constexpr int TM_RING_WORDS = 256 * TM_KW + 64 * TM_KW * 4;  // A: 256 rows x 2 words, B: 128 rows x 4 words
constexpr size_t TM_SMEM_BYTES = 2 * TM_STAGE_BYTES + TM_RING * TM_RING_WORDS * 8 + 1024;
static_assert(TM_SMEM_BYTES <= 227 * 1024, "tc_mul shared memory");

struct TcMulArgs {
    uint64_t *C;
    int64_t ldc;
    const uint64_t *A;
    int64_t lda;
    const uint64_t *B;
    int64_t ldb;
    int64_t m, k, n;
    int32_t *err;
};

namespace {

// 4 bits -> 4 FP8 bytes (1.0 = 0x38 where the bit is set)
__device__ __forceinline__ uint32_t nib_fp8_tc(uint32_t b)
{
    uint32_t t = (b & 15u) * 0x01010101u;
    t &= 0x08040201u;
    t = ((t + 0x7F7F7F7Fu) & 0x80808080u) >> 7;
    return t * 0x38u;
}

// Byte offset of (row, 16-byte K group j) in the core-matrix layout of a
// 128-byte-per-row chunk: K-direction stride 128 bytes, 8-row groups 1024 apart.
__device__ __forceinline__ uint32_t core_off8(int row, int j)
{
    return (uint32_t)(((row >> 3) * 8 + j) * 128 + (row & 7) * 16);
}

// 32 bits -> K groups j0 and j0 + 1 (16 bytes each) of a row in that layout
__device__ __forceinline__ void expand_store_half(uint8_t *tile, int row, int j0, uint32_t bits)
{
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const uint32_t h = bits >> (16 * q);
        uint4 v;
        v.x = nib_fp8_tc(h);
        v.y = nib_fp8_tc(h >> 4);
        v.z = nib_fp8_tc(h >> 8);
        v.w = nib_fp8_tc(h >> 12);
        *reinterpret_cast<uint4 *>(tile + core_off8(row, j0 + q)) = v;
    }
}

__device__ __forceinline__ void cp_async8_tc(void *dst, const void *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr(dst)), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit_tc() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_tc() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

}  // namespace

__global__ void __launch_bounds__(TM_THREADS, 1) tc_mul_kernel(TcMulArgs a)
{
    extern __shared__ __align__(1024) uint8_t tm_smem[];
    __shared__ __align__(8) uint64_t sfree[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint8_t *stage0 = tm_smem + ((1024u - (saddr(tm_smem) & 1023u)) & 1023u);
    uint64_t *ring = reinterpret_cast<uint64_t *>(stage0 + 2 * TM_STAGE_BYTES);

    if (tid == 0) {
        mbar_init(&sfree[0], 1);
        mbar_init(&sfree[1], 1);
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(&tmem_base)),
                     "r"(TM_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    const int64_t m = a.m, k = a.k, n = a.n;
    const int64_t Wc = (n + 63) >> 6;
    const int64_t KC = (k + TM_KB - 1) / TM_KB;
    const int64_t NTX = (n + 255) >> 8, NTY = (m + 255) >> 8;
    const int64_t T = NTX * NTY;
    // work split per chunk: thread t expands word t & 1 of A row t / 2 (K
    // groups 4 (t & 1) .. + 3); warp w transposes two 32 x 32 blocks of B --
    // generator rows 64 (w & 1) + 32 h (h = 0, 1), columns 64 (w / 4) +
    // 32 ((w / 2) & 1) .. -- and each lane expands one column's 32 bits per
    // block into K groups 4 (w & 1) + 2 h and up
    const int arow = tid >> 1, aword = tid & 1;
    const int bword = warp >> 2, bchalf = (warp >> 1) & 1, bkq = warp & 1;
    int64_t g = 0;                                   // chunks issued by this CTA so far
    for (int64_t t = blockIdx.x; t < T && KC > 0; t += gridDim.x) {
        const int64_t tx = t / NTY, ty = t - tx * NTY;   // neighbouring CTAs share a column tile of B
        const int64_t row0 = ty * 256, wb = tx * 4;
        // operand bits, chunk kc in ring slot kc % TM_RING: A rows (256 x
        // TM_KW words) then B's 128 generator rows x 4 words, copied by
        // cp.async TM_RING - 1 chunks ahead of their expansion
        const int64_t ia = row0 + arow;
        auto issue = [&](int64_t kc) {
            uint64_t *slot = ring + (kc % TM_RING) * TM_RING_WORDS;
            if (kc < KC) {
                {                                            // A: row row0 + t / 2, word TM_KW kc + (t & 1)
                    const int64_t r = row0 + (tid >> 1), w = TM_KW * kc + (tid & 1);
                    const bool ok = r < m && 64 * w < k;
                    cp_async8_tc(slot + tid, a.A + (ok ? r * a.lda + w : 0), ok);
                }
                {                                            // B: generator row 128 kc + t / 4, word wb + (t & 3)
                    const int64_t r = (int64_t)TM_KB * kc + (tid >> 2), w = wb + (tid & 3);
                    const bool ok = r < k && w < Wc;
                    cp_async8_tc(slot + 256 * TM_KW + tid, a.B + (ok ? r * a.ldb + w : 0), ok);
                }
            }
            cp_async_commit_tc();
        };
        for (int q = 0; q < TM_RING - 1; ++q) issue(q);
        cp_async_wait_tc<TM_RING - 2>();                     // chunk 0 has landed (this thread's part)
        __syncthreads();
        for (int64_t kc = 0; kc < KC; ++kc) {
            const int st = (int)(g & 1);
            const uint64_t *slot = ring + (kc % TM_RING) * TM_RING_WORDS;
            uint64_t va = slot[tid];                         // word aword of A row arow
            const int64_t rem = k - 64 * (TM_KW * kc + aword);
            if (rem < 64) va = rem <= 0 ? 0ull : (va & ((1ull << rem) - 1ull));
            if (ia >= m) va = 0;
            // the MMAs of chunk g - 2 read this stage: wait until they are done
            if (g >= 2 && !mbar_wait_bounded(&sfree[st], (uint32_t)(((g >> 1) - 1) & 1))) {
                s_abort = 1;
                if (a.err) atomicExch(a.err, 4);         // GF2_ETIMEOUT
            }
            uint8_t *sA = stage0 + st * TM_STAGE_BYTES;
            uint8_t *sB = sA + 2 * TM_A_BYTES;
            uint8_t *tA = sA + (arow >> 7) * TM_A_BYTES;
            expand_store_half(tA, arow & 127, 4 * aword, (uint32_t)va);
            expand_store_half(tA, arow & 127, 4 * aword + 2, (uint32_t)(va >> 32));
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int kr = 64 * bkq + 32 * hh + lane;    // generator row within the chunk
                const uint32_t xb = (uint32_t)(slot[256 * TM_KW + kr * 4 + bword] >> (32 * bchalf));
                const unsigned col = transpose32_tc(xb); // lane c: one column over 32 generator rows
                expand_store_half(sB, bword * 64 + bchalf * 32 + lane, 4 * bkq + 2 * hh, col);
            }
            issue(kc + TM_RING - 1);                     // into the slot chunk kc - 1 used
            cp_async_wait_tc<TM_RING - 2>();             // chunk kc + 1 has landed
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (s_abort) break;
            if (tid == 0) {
                tc_fence_after();
                const uint32_t a0 = saddr(sA), a1 = a0 + TM_A_BYTES, b0 = saddr(sB);
#pragma unroll
                for (int ks = 0; ks < TM_KB / 32; ++ks) {
                    const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                    mma_f8(tmem, smem_desc(a0 + ks * 256, 128, 1024), smem_desc(b0 + ks * 256, 128, 1024), acc);
                    mma_f8(tmem + 256, smem_desc(a1 + ks * 256, 128, 1024), smem_desc(b0 + ks * 256, 128, 1024),
                           acc);
                }
                mma_commit(&sfree[st]);
            }
            ++g;
        }
        cp_async_wait_tc<0>();
        if (s_abort) break;
        // every MMA of the tile has completed once the last chunk's commit has
        if (!mbar_wait_bounded(&sfree[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1))) {
            s_abort = 1;
            if (a.err) atomicExch(a.err, 4);
        }
        __syncthreads();
        if (s_abort) break;
        tc_fence_after();
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. of
        // accumulator (w / 4) % 2, columns 128 (w / 8) .. + 127
        const int quad = warp & 3, accn = (warp >> 2) & 1, chalf = warp >> 3;
        const int64_t i = row0 + 128 * accn + 32 * quad + lane;
#pragma unroll 1
        for (int cb = 0; cb < 4; cb += 2) {
            uint32_t v0[32], v1[32];
            const uint32_t base = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(256 * accn + 128 * chalf);
            tmem_ld32(base + (uint32_t)(cb * 32), v0);
            tmem_ld32(base + (uint32_t)((cb + 1) * 32), v1);
            uint32_t p0 = 0, p1 = 0;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                p0 |= (__float_as_uint(__uint_as_float(v0[q]) + 8388608.0f) & 1u) << q;
                p1 |= (__float_as_uint(__uint_as_float(v1[q]) + 8388608.0f) & 1u) << q;
            }
            const int64_t w = wb + 2 * chalf + cb / 2;
            if (i < m && w < Wc) a.C[i * a.ldc + w] ^= ((uint64_t)p1 << 32) | p0;
        }
        tc_fence_before();
        __syncthreads();                             // tensor memory read out before the next tile's MMAs
        tc_fence_after();
    }
    if (s_abort && g > 0) mbar_wait_bounded(&sfree[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1));
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TM_TMEM_COLS));
}

cudaError_t launch_tc_mul(cudaStream_t st, uint64_t *C, int64_t ldc, const uint64_t *A, int64_t lda, const uint64_t *B,
                          int64_t ldb, int64_t m, int64_t k, int64_t n, int32_t *err, int num_sms)
{
    static bool attr = false;
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(tc_mul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TM_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    TcMulArgs a{C, ldc, A, lda, B, ldb, m, k, n, err};
    const int64_t tiles = ((n + 255) >> 8) * ((m + 255) >> 8);
    const int grid = (int)std::min<int64_t>(num_sms, std::max<int64_t>(tiles, 1));
    tc_mul_kernel<<<grid, TM_THREADS, TM_SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_update_tc(cudaStream_t st, const UpdArgs &a, int num_sms)
{
    const int grid = (a.grid > 0 && a.grid < num_sms) ? a.grid : num_sms;
    tc_update_kernel<<<grid, TC_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gf2
