// kernels_update_tma.cu -- the TMA-staged, warp-specialised form of the
// tabulated trailing update (GF2_OPT_TMA_UPDATE), and the encoding of its
// tensor map.
#include "async_dev.cuh"
#include "tables_dev.cuh"

#include <cuda.h>

namespace gf2 {

// ----------------------------------------------------------------------------
// TMA form (16-byte aligned rows, even leading dimension, a tensor map of A):
// warp-specialised.  The same paired walk over (tile pair x rows) as
// update_pipe_kernel, in units of 256-row batches.  One producer warp moves
// the batches' 64-byte row tiles between HBM and shared memory with TMA
// (one box load per batch into one of five stages, and one box store once
// the consumers release it); sixteen consumer warps do the table lookups in
// shared memory and never wait for one another except when the column tile
// changes.  Row data then never passes through the LSU as global requests
// (ncu on update_pipe_kernel: about 30 of its 73% L1 data-pipe wavefronts
// were the global row loads and stores).  Each consumer thread prefetches the
// 8-byte table indices of its rows three batches ahead.  The quad of threads
// on a row reads its 16-byte pieces of two consecutive rows per quarter-warp,
// 128 contiguous bytes, so the unswizzled stage is conflict-free.  Batches
// that end past the row range, and the first tile when it starts left of the
// update range, are written back by the consumers, word by word in range,
// instead of the TMA store.
constexpr int TMA_ROWS = 256;                        // rows per batch = one box
constexpr int TMA_STAGE_BYTES = TMA_ROWS * TW * 8;   // 16 KiB
constexpr int TMA_STAGES = 5;                       // 3 loads in flight, 1 updated, 1 stored
constexpr int WS_CONSUMER_WARPS = UPD_THREADS / 32;  // 16
constexpr int WS_THREADS = UPD_THREADS + 32;         // + the producer warp
constexpr size_t TMA_SMEM_BYTES = (size_t)TAB_WORDS * 8 + (size_t)TMA_STAGES * TMA_STAGE_BYTES + 128;

__device__ __forceinline__ void mbar_arrive_cta(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(UPD_THREADS) : "memory"); }

__global__ void __launch_bounds__(WS_THREADS, 1)
update_tma_kernel(UpdArgs a, const __grid_constant__ TensorMap2D tm)
{
    extern __shared__ __align__(128) unsigned char upd_smem[];
    unsigned char *sbase = upd_smem + ((128u - (smem_u32(upd_smem) & 127u)) & 127u);
    uint64_t *T = reinterpret_cast<uint64_t *>(sbase);
    unsigned char *stage = sbase + (size_t)TAB_WORDS * 8;
    __shared__ __align__(8) uint64_t full[TMA_STAGES], empty[TMA_STAGES];
    __shared__ const uint64_t *sGen[KS];
    __shared__ volatile int s_abort;

    int64_t row_lo, row_hi, w_lo;
    const int64_t W = a.W;
    int64_t r = 0;
    int maxpos = -1, nS = 0;
    const StripeDesc *d = a.desc;
    if (a.mode == UPD_PLE) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        r = d->r;
        row_lo = r;
        row_hi = a.m;
        w_lo = (d->c >> 6) + (a.first_off > 0 ? a.first_off : 1);
        maxpos = d->maxpos;
        nS = d->nS;
        if (threadIdx.x < KS)
            sGen[threadIdx.x] = (threadIdx.x < rbar) ? a.S + threadIdx.x * a.ldS : nullptr;
    } else if (a.mode == UPD_RREF) {
        const int rbar = d->rbar;
        if (rbar == 0) return;
        row_lo = a.row_lo;                    // 0, or the first row of a block's own RREF
        row_hi = d->r;
        w_lo = max((int64_t)(d->c >> 6), a.w_lo);  // a.w_lo > 0: only a right part of the row
        if (threadIdx.x < KS) sGen[threadIdx.x] = nullptr;
        __syncthreads();
        if (threadIdx.x < rbar) sGen[d->qbar[threadIdx.x]] = a.A + (d->r + threadIdx.x) * a.ld;
    } else {
        row_lo = a.row_lo;
        row_hi = a.row_hi;
        w_lo = a.w_lo;
        if (threadIdx.x < KS)
            sGen[threadIdx.x] = (threadIdx.x < a.gen_count) ? a.B + threadIdx.x * a.ldb : nullptr;
    }
    __syncthreads();

    if (a.mode == UPD_PLE && a.left_copies) {
        for (int k = blockIdx.x; k < nS; k += gridDim.x) {
            const uint64_t *src = a.S + (int64_t)k * a.ldS;
            uint64_t *dst = a.A + (r + d->S_off[k]) * a.ld;
            for (int64_t w = threadIdx.x; w < w_lo; w += blockDim.x) dst[w] = src[w];
        }
    }

    const int64_t R = row_hi - row_lo;
    if (R <= 0 || w_lo >= W) return;
    const int64_t a0 = w_lo / TW, a1 = (W + TW - 1) / TW;
    const int64_t NT = a1 - a0;
    const int64_t NTP = (NT + 1) / 2;
    const int64_t tp_lo = min(a.tp_lo, NTP);
    const int64_t tp_hi = (a.tp_hi < 0) ? NTP : min(a.tp_hi, NTP);
    if (tp_lo >= tp_hi) return;
    const int npairs = gridDim.x >> 1;
    const int pj = blockIdx.x >> 1, half = blockIdx.x & 1;
    if (pj >= npairs) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.bytes) {
        const int64_t wl = max(w_lo, (a0 + 2 * tp_lo) * TW);
        const int64_t wh = min(W, (a0 + 2 * tp_hi) * TW);
        atomicAdd(a.bytes, (unsigned long long)(R * (wh - wl) * 16));
    }
    const int64_t NB = (R + TMA_ROWS - 1) / TMA_ROWS;
    const int64_t U = (tp_hi - tp_lo) * NB;
    const int64_t u_beg = U * pj / npairs;
    int64_t u_end = U * (pj + 1) / npairs;
    if (2 * (tp_hi - 1) + half >= NT) u_end = min(u_end, (tp_hi - 1 - tp_lo) * NB);   // odd last pair
    const int64_t nunits = u_end - u_beg;
    if (nunits <= 0) return;

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int st = 0; st < TMA_STAGES; ++st) {
            mbar_init_cta(&full[st], 1);
            mbar_init_cta(&empty[st], WS_CONSUMER_WARPS);
        }
        mbar_init_fence();
        s_abort = 0;
    }
    __syncthreads();                                  // the last block-wide barrier

    auto unit_tile = [&](int64_t u) { return 2 * (tp_lo + u / NB) + half; };
    auto unit_row0 = [&](int64_t u) { return row_lo + (u % NB) * TMA_ROWS; };
    auto unit_x = [&](int64_t u) { return (a0 + unit_tile(u)) * TW; };
    auto unit_tma_out = [&](int64_t u) { return unit_x(u) >= w_lo && unit_row0(u) + TMA_ROWS <= row_hi; };

    if (tid >= UPD_THREADS) {
        // ---------------- producer warp: lane 0 issues every copy
        if (tid != UPD_THREADS) return;
        // Loads run up to TMA_STAGES - 2 batches ahead of the batch being
        // released, so the stage a load reuses was released (and its store
        // committed) at least two batches earlier: its store has normally
        // finished reading shared memory and the wait below does not block.
        int64_t k_load = 0, issued = 0;
        for (int64_t k_rel = 0; k_rel <= nunits; ++k_rel) {
            const int64_t lim = min(nunits, k_rel + TMA_STAGES - 1);
            while (k_load < lim) {
                const int st = (int)(k_load % TMA_STAGES);
                if (k_load >= TMA_STAGES) {
                    const int64_t j = k_load - TMA_STAGES;      // the batch that held this stage
                    if (unit_tma_out(u_beg + j)) {
                        int later = 0;                          // stores committed after batch j's
                        for (int64_t t = j + 1; t < k_rel; ++t) later += unit_tma_out(u_beg + t) ? 1 : 0;
                        if (later <= 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
                        else if (later == 1) asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
                        else if (later == 2) asm volatile("cp.async.bulk.wait_group.read 2;\n" ::: "memory");
                        else asm volatile("cp.async.bulk.wait_group.read 3;\n" ::: "memory");
                    }
                }
                mbar_expect_tx(&full[st], TMA_STAGE_BYTES);
                tma_load_2d(stage + st * TMA_STAGE_BYTES, &tm, (int)unit_x(u_beg + k_load),
                            (int)unit_row0(u_beg + k_load), &full[st]);
                issued = ++k_load;
            }
            if (k_rel == nunits) break;
            const int st = (int)(k_rel % TMA_STAGES);
            if (s_abort || !mbar_wait_limited(&empty[st], (uint32_t)((k_rel / TMA_STAGES) & 1))) {
                s_abort = 1;
                if (a.err) atomicExch(a.err, 4);              // GF2_ETIMEOUT
                break;
            }
            if (unit_tma_out(u_beg + k_rel)) {
                tma_store_2d(&tm, (int)unit_x(u_beg + k_rel), (int)unit_row0(u_beg + k_rel),
                             stage + st * TMA_STAGE_BYTES);
                bulk_commit();
            }
        }
        bulk_wait_all();                              // stores complete before the kernel ends
        if (s_abort) {
            // let the box loads still in flight land before the CTA's shared memory goes away
            for (int64_t k = (issued > TMA_STAGES ? issued - TMA_STAGES : 0); k < issued; ++k)
                mbar_wait_limited(&full[k % TMA_STAGES], (uint32_t)((k / TMA_STAGES) & 1));
        }
        return;
    }

    // ---------------- consumer warps
    const int lane = tid & 31;
    const int rs = tid >> 2, qd = tid & 3, rho = rs & 1;
    constexpr int SLOTS = UPD_THREADS / 4;
    constexpr int RPB = TMA_ROWS / SLOTS;             // rows per thread and batch (2)
    auto load_ix = [&](int64_t k, uint64_t (&ix)[RPB]) {
#pragma unroll
        for (int q = 0; q < RPB; ++q) {
            ix[q] = 0;
            if (k < nunits) {
                const int64_t i = unit_row0(u_beg + k) + q * SLOTS + rs;
                if (i < row_hi) ix[q] = __ldg(a.idx + i * a.idx_stride);
            }
        }
    };
    uint64_t ix0[RPB], ix1[RPB], ix2[RPB], ix3[RPB];
    load_ix(0, ix0);
    load_ix(1, ix1);
    load_ix(2, ix2);
    int64_t cur_tile = -1;
    for (int64_t k = 0; k < nunits; ++k) {
        const int st = (int)(k % TMA_STAGES);
        const int64_t u = u_beg + k;
        const int64_t tile = unit_tile(u), y0 = unit_row0(u);
        const int64_t wbase = (a0 + tile) * TW;
        load_ix(k + 3, ix3);                          // three batches ahead
        if (tile != cur_tile) {
            consumers_sync();                         // every consumer is done with the old tables
            build_tables(T, sGen, wbase, W);
            consumers_sync();
            cur_tile = tile;
        }
        bool ok = !s_abort;
        if (ok && !mbar_wait_limited(&full[st], (uint32_t)((k / TMA_STAGES) & 1))) {
            s_abort = 1;
            if (a.err) atomicExch(a.err, 4);
            ok = false;
        }
        ok = __all_sync(0xffffffffu, ok);
        const bool tma_out = unit_tma_out(u);
        if (ok) {
            const int64_t w0 = wbase + 2 * qd;
            const bool lo_in = w0 >= w_lo && w0 < W;
            const bool hi_in = w0 + 1 >= w_lo && w0 + 1 < W;
            unsigned char *sb = stage + st * TMA_STAGE_BYTES;
            const uint64_t *Tq = T + 2 * qd;
#pragma unroll
            for (int q = 0; q < RPB; ++q) {
                const int y = q * SLOTS + rs;
                const int64_t i = y0 + y;
                ulonglong2 *cell = reinterpret_cast<ulonglong2 *>(sb + y * (TW * 8) + qd * 16);
                ulonglong2 v = *cell;
                if (a.mode == UPD_PLE && i - r <= maxpos && i < row_hi) {
                    const int mv = a.map[i];
                    if (mv >= 0 && (mv >> 8) == a.stripe) {   // staged row: its content sits in S
                        const uint64_t *sp = a.S + (int64_t)(mv & 255) * a.ldS;
                        v.x = lo_in ? sp[w0] : 0ull;
                        v.y = hi_in ? sp[w0 + 1] : 0ull;
                    }
                }
                const uint64_t e8 = ix0[q];
#pragma unroll
                for (int uu = 0; uu < NTAB; ++uu) {
                    const int tau = uu ^ rho;
                    const int e = (int)((e8 >> (8 * tau)) & 255ull);
                    const ulonglong2 tv = *reinterpret_cast<const ulonglong2 *>(
                        Tq + (tau >> 1) * (256 * TAB_LINE) + e * TAB_LINE + (tau & 1) * TW);
                    v.x ^= tv.x;
                    v.y ^= tv.y;
                }
                if (tma_out) {
                    *cell = v;
                } else if (i < row_hi) {
                    uint64_t *dst = a.A + i * a.ld;
                    if (lo_in && hi_in) {
                        *reinterpret_cast<ulonglong2 *>(dst + w0) = v;
                    } else {
                        if (lo_in) dst[w0] = v.x;
                        if (hi_in) dst[w0 + 1] = v.y;
                    }
                }
            }
            if (tma_out) fence_proxy_async_smem();    // the producer's store reads these writes
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_cta(&empty[st]);
#pragma unroll
        for (int q = 0; q < RPB; ++q) {
            ix0[q] = ix1[q];
            ix1[q] = ix2[q];
            ix2[q] = ix3[q];
        }
    }
}

cudaError_t setup_update_tma_kernel()
{
    return cudaFuncSetAttribute(update_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TMA_SMEM_BYTES);
}

cudaError_t launch_update_tma(cudaStream_t st, const UpdArgs &a, int grid)
{
    update_tma_kernel<<<grid, WS_THREADS, TMA_SMEM_BYTES, st>>>(a, *a.tmap);
    return cudaGetLastError();
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn()
{
    // the driver's encoder, looked up once through the runtime (no libcuda link)
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

}  // namespace

static_assert(sizeof(CUtensorMap) == sizeof(TensorMap2D), "tensor map size");

bool encode_row_tiles(TensorMap2D *out, const uint64_t *A, int64_t m, int64_t W, int64_t ld)
{
    if (!out || !A || ((uintptr_t)A & 15u) || (ld & 1) || W < 2 * TW || m < TMA_ROWS ||
        m > (int64_t(1) << 30) || W > (int64_t(1) << 30))
        return false;
    const EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)m};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
    const cuuint32_t box[2] = {(cuuint32_t)TW, (cuuint32_t)TMA_ROWS};
    const cuuint32_t estr[2] = {1, 1};
    return fn(reinterpret_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t *>(A), dims,
              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Expanded FP4 operand of the own GEMM (kernels_gemm_f4.cu): `rows` rows of
// `rowb` bytes, boxes of box_rows rows x 128 bytes with the 128-byte swizzle
// the MMA descriptors expect; the caller pads so that the tensor is at least
// one box in each dimension.  Out-of-range boxes read zeros.
bool encode_f4_operand(TensorMap2D *out, const uint8_t *base, int64_t rows, int64_t rowb, int box_rows)
{
    if (!out || !base || ((uintptr_t)base & 15u) || (rowb & 15) || rowb < 128 || rows < box_rows ||
        box_rows < 1 || box_rows > 256 || rows > (int64_t(1) << 31) - 1 || rowb > (int64_t(1) << 31) - 1)
        return false;
    const EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)rowb, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)rowb};
    const cuuint32_t box[2] = {128u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(reinterpret_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(base),
              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


}  // namespace gf2
