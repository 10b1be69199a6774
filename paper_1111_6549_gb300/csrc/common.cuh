// common.cuh -- shared definitions of the sm_103a GF(2) elimination kernels.
//
// Data layout: row-major bit-packed matrices, column j = bit (j % 64) of
// word j / 64.  The block-iterative PLE (Algorithm 2) walks the columns in
// stripes of KS = 64 columns (one word per row), so every stripe starts on a
// word boundary.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace gf2 {

// ---- programmatic dependent launch (PDL)
// A kernel of this library starts with pdl_wait() -- it returns once the
// kernel launched before it on the stream has completed and its memory
// operations are visible (at once when there is none, or when the kernel was
// launched without the attribute) -- and pdl_trigger(), which lets the next
// kernel on the stream be scheduled while this one runs (its CTAs then sit in
// their own pdl_wait()).  Only the waiting is needed for correctness; the
// early scheduling hides the launch latency between dependent kernels.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Launches made by the calling thread carry the PDL attribute while this is
// set (the handle's GF2_OPT_PDL, set for the duration of each call).
extern thread_local bool g_pdl;

template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args &&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = g_pdl ? attr : nullptr;
    cfg.numAttrs = g_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int KS = 64;            // stripe width in columns (one uint64 word)
constexpr int SMAX = 2 * KS;      // rows staged per stripe: pivot rows + displaced rows
constexpr int TW = 8;             // update tile width in words (64 bytes per row)
constexpr int NTAB = KS / 8;      // 8-bit tables per stripe
constexpr int TAB_LINE = 2 * TW;  // words per shared-memory line (two tables interleaved)
constexpr int TAB_WORDS = (NTAB / 2) * 256 * TAB_LINE;  // 16384 words = 128 KiB
// Wide form of the update: 128-byte tiles, eight 7-bit tables + one 8-bit
// table per stripe (entry e of table t at entry offset 128 t + e).
constexpr int WT = 16;            // wide tile width in words (128 bytes per row)
constexpr int WNTAB = 9;
constexpr int WIDE_TAB_WORDS = (8 * 128 + 256) * WT;    // 20480 words = 160 KiB
constexpr int UPD_THREADS = 512;
constexpr int UPD_ROWS_PER_THREAD = 4;
constexpr int PANEL_THREADS = 512;
constexpr int PANEL_WIN = 128;    // fast panel window: rows held bit-sliced by one warp

// Per-stripe record written by the panel kernel and read by the later
// kernels of the stripe (and by the RREF recovery).
struct StripeDesc {
    int64_t r;          // rank before this stripe (first row position of the stripe)
    int32_t rbar;       // pivots found in the stripe
    int32_t c;          // first column of the stripe
    int32_t nS;         // staged rows: [0, rbar) pivot rows, then displaced rows
    int32_t maxpos;     // largest position offset (from r) of a staged row
    int32_t tier;       // 1: warp window path, 2: block-wide path
    int32_t pad;
    uint64_t E11[KS];   // pivot rows' stripe word after elimination (echelon)
    uint64_t L11[KS];   // L coefficients of pivot rows w.r.t. earlier pivots (bit q < p)
    uint64_t Linv[KS];  // rows of L11^-1 (unit lower triangular)
    uint64_t Minv[KS];  // rows of U11^-1, U11 = E11 on the pivot columns (unit upper triangular)
    int32_t S_off[SMAX];  // staged row k -> position offset from r
    int64_t S_src[SMAX];  // staged row k -> physical row copied from
    uint8_t qbar[KS];     // pivot column offsets inside the stripe
};

// One matrix of the batched entry point (same layout as gf2_desc).
struct gf2_batch_item {
    uint64_t *A;
    int64_t m, n, ld_words;
    int64_t *P;
    int64_t *Q;
    int64_t *rank;
};
constexpr int64_t BATCH_MAX_ROWS = 4096;   // larger matrices take the single-matrix path
constexpr int64_t BATCH_MAX_COLS = 4096;

// Tuning of the batched kernel.  A matrix's size class is set by max(m, n):
// <= 128, <= 256, <= 512, <= 1024, <= 2048, <= 4096.  Each class runs one
// table configuration: k-bit tables (64 / k of them per stripe) over tiles of
// BW words.
constexpr int BATCH_CLASSES = 6;
constexpr int BATCH_CONFIGS = 5;
constexpr int BATCH_CFG_K[BATCH_CONFIGS] = {8, 8, 4, 4, 4};
constexpr int BATCH_CFG_BW[BATCH_CONFIGS] = {2, 1, 1, 2, 4};
constexpr int BATCH_CFG_DEFAULT = 0;
struct BatchTune {
    int8_t cfg[BATCH_CLASSES];
};
__host__ __device__ inline int batch_size_class(int64_t m, int64_t n)
{
    const int64_t s = m > n ? m : n;
    return s <= 128 ? 0 : s <= 256 ? 1 : s <= 512 ? 2 : s <= 1024 ? 3 : s <= 2048 ? 4 : 5;
}

// Scratch of the block-wide panel path: one entry per remaining row.
// Entries are the rows whose stripe word is nonzero, in position order.
struct PanelScratch {
    uint64_t *val;   // stripe word, eliminated eagerly
    uint64_t *lb;    // L coefficient bits
    int32_t *src;    // row offset (from r) whose content sits in this entry
    int32_t *pos;    // current position offset of the entry (-1: taken as a pivot or retired)
};

enum UpdMode { UPD_PLE = 0, UPD_RREF = 1, UPD_MUL = 2, UPD_M4RI = 3 };

struct UpdArgs {
    int mode;
    uint64_t *A;               // destination rows (and default source)
    int64_t ld;
    int64_t m;                 // PLE/RREF: rows of A
    int64_t W;                 // words per row to process (exclusive upper bound)
    const StripeDesc *desc;    // PLE/RREF: the stripe record
    int stripe;
    const uint64_t *S;         // PLE: staged rows
    int64_t ldS;
    const int32_t *map;        // PLE: position -> stripe * 256 + staged slot, or -1
    const uint64_t *idx;       // table index per row (row i at idx[i * idx_stride])
    int64_t idx_stride;
    const uint64_t *B;         // MUL: generator rows B + g * ldb; M4RI: the reduced pivot rows
    int64_t ldb;
    int64_t gen_count;         // MUL: number of generator rows (<= 64)
    int64_t row_lo, row_hi;    // MUL: rows to update; RREF: row_lo = first row updated (rows end at the block)
    int64_t w_lo;              // MUL: first word to update
    unsigned long long *bytes; // algorithmic bytes counter (may be null)
    int64_t tp_lo, tp_hi;      // tile pairs [tp_lo, tp_hi) of the column range (tp_hi < 0: all)
    int left_copies;           // PLE: also write the staged rows' left parts
    int grid;                  // CTAs to launch (0: one per SM)
    int32_t *err;              // device error word (bounded waits that expire), may be null
    const struct TensorMap2D *tmap;  // TMA descriptor of A's rows (null: plain loads and stores)
    int64_t W_full;            // PLE: row width; staged rows also get words [W, W_full) (0: none)
    int wide;                  // aligned rows: 128-byte tiles with nine tables (else paired 64-byte tiles)
    int naive;                 // plain baseline: generator rows added one by one, no tables
    int first_off;             // PLE: first updated word = stripe word + first_off (0: 1)
    // RREF passes with the block reduction fused in (wide table kernel only):
    // each CTA forms the stripe's reduced pivot rows G = U11^-1 rows for its
    // tiles in shared memory and writes them to gbuf_w (row t of the stripe
    // at gbuf_w + t * ldg); the pass also writes the previous pass's G from
    // gbuf_r back into that stripe's pivot rows (flush_desc, may be null)
    // and takes the next pass's table index -- the stripe word of rows
    // [row_lo, r) of snap_desc -- into idx_next (snap_desc may be null).
    int rref_fused;
    uint64_t *gbuf_w;
    const uint64_t *gbuf_r;
    int64_t ldg;
    const StripeDesc *flush_desc;
    const StripeDesc *snap_desc;
    uint64_t *idx_next;
    int64_t skip_lo, skip_hi;  // words [skip_lo, skip_hi) may be left out (zero in every row
                               // involved); the pipelined table kernels use it
};

// A CUtensorMap (128 bytes) kept opaque outside the files that use TMA.
struct alignas(64) TensorMap2D {
    unsigned char bytes[128];
};
// Encode the TMA descriptor of an m x W word matrix with row stride ld words
// for the update kernel's 64-byte x 256-row boxes; false when A is not
// eligible (base not 16-byte aligned, odd ld, fewer than 16 words or 256 rows).
bool encode_row_tiles(TensorMap2D *out, const uint64_t *A, int64_t m, int64_t W, int64_t ld);

// ---- launchers (host side, defined in the .cu files) ----
cudaError_t launch_init_ple(cudaStream_t st, int64_t *P, int64_t *Q, int64_t m, int64_t qn,
                            int32_t *map, int64_t *r_dev, int num_sms);
// The panel kernel also writes the bases of the prep kernel's lookup tables
// (3 x 64 words by stripe column, at the start of the PREP_TAB_BYTES reserved
// per stripe parity) to ptab when it is not null; the prep builds its tables
// in shared memory from them.
constexpr int PREP_TAB_WORDS = 8 * 256;
constexpr size_t PREP_TAB_BYTES = 3 * PREP_TAB_WORDS * sizeof(uint64_t);
// prev_map / prev_S (may be null): the previous stripe's row map and staged
// rows, read for the rows its swaps moved while its update may still run.
cudaError_t launch_panel(cudaStream_t st, uint64_t *A, int64_t m, int64_t ld, int64_t npiv, int s,
                         StripeDesc *descs, int64_t *r_dev, int64_t *P, int64_t *Q, int32_t *map,
                         PanelScratch gs, int32_t *fallbacks, uint64_t *ptab, const int32_t *prev_map = nullptr,
                         const uint64_t *prev_S = nullptr, int64_t ldS = 0);
// next_word >= 0: the prep also applies the stripe's update to that word of
// every row (the next stripe's word, for its panel to start early; the
// update kernel then starts one word later, UpdArgs::first_off = 2).
cudaError_t launch_prep(cudaStream_t st, uint64_t *A, int64_t m, int64_t ld, int64_t W, int s,
                        StripeDesc *descs, const int32_t *map, uint64_t *S, int64_t ldS,
                        uint64_t *IDX, int32_t *err, const uint64_t *ptab, int num_sms, int64_t next_word = -1);
cudaError_t setup_update_kernel();
cudaError_t setup_prep_kernel();
cudaError_t launch_update(cudaStream_t st, const UpdArgs &a, int num_sms);
// the fused RREF stripe pass (UpdArgs::rref_fused; kernels_rref_pass.cu)
cudaError_t setup_rref_pass_kernel();
cudaError_t launch_rref_pass(cudaStream_t st, const UpdArgs &a, int num_sms);
bool update_vectorised(const UpdArgs &a);   // true when the paired, pipelined form runs
cudaError_t launch_update_tc(cudaStream_t st, const UpdArgs &a, int num_sms);
cudaError_t launch_tc_mul(cudaStream_t st, uint64_t *C, int64_t ldc, const uint64_t *A, int64_t lda, const uint64_t *B,
                          int64_t ldb, int64_t m, int64_t k, int64_t n, int32_t *err, int num_sms);
cudaError_t setup_update_tma_kernel();
cudaError_t launch_update_tma(cudaStream_t st, const UpdArgs &a, int grid);   // a.tmap must be set
// compact RREF recovery: rows i < r rewritten as the identity on their pivot
// columns Q and the reduced non-pivot bits C (kwn words per row) elsewhere
cudaError_t launch_rref_scatter(cudaStream_t st, uint64_t *A, int64_t ld, int64_t W, int64_t r, const int64_t *Q,
                                const uint64_t *C, int64_t kwn, const uint64_t *npmask, const int64_t *npstart,
                                int num_sms);
cudaError_t launch_rref_lclear(cudaStream_t st, uint64_t *A, int64_t m, int64_t W, int64_t ld,
                               const int64_t *r_dev, int num_sms);
cudaError_t launch_rref_prep(cudaStream_t st, uint64_t *A, int64_t ld, int64_t W, int s,
                             const StripeDesc *descs, uint64_t *IDX, int64_t m, int num_sms);
// The fused RREF passes' bookends: flush_desc (may be null): the stripe's
// reduced pivot rows from gbuf into A over the words [c >> 6, W) except
// [skip_lo, skip_hi); snap_desc (may be null): the stripe word of rows
// [row_lo, r) into idx.
cudaError_t launch_rref_aux(cudaStream_t st, uint64_t *A, int64_t ld, const StripeDesc *flush_desc,
                            const uint64_t *gbuf, int64_t ldg, int64_t W, int64_t skip_lo, int64_t skip_hi,
                            const StripeDesc *snap_desc, uint64_t *idx, int64_t row_lo, int num_sms);
cudaError_t launch_copy_rank(cudaStream_t st, const int64_t *r_dev, int64_t *rank_dev);
// GF(2) product through the own FP4 tcgen05 GEMM (kernels_gemm_f4.cu): A4
// a_rows >= max(m, 256) and B4t b_rows >= max(n, 192) rows of kp / 2 bytes
// each (expanded operands, zero past m / n rows; kp a multiple of 256);
// C (m x n bits) ^= the parities of A4 B4t^T.
cudaError_t launch_gemm_f4(cudaStream_t st, uint64_t *C, int64_t ldc, const uint8_t *A4, int64_t a_rows,
                           const uint8_t *B4t, int64_t b_rows, int64_t m, int64_t n, int64_t kp, int32_t *err,
                           int num_sms);
bool encode_f4_operand(TensorMap2D *out, const uint8_t *base, int64_t rows, int64_t rowb, int box_rows);
// GF(2) product through a library FP4 / FP8 GEMM (kernels_gemm.cu)
cudaError_t launch_expand_rows(cudaStream_t st, int fmt, const uint64_t *A, int64_t lda, int64_t rows, int64_t k0,
                               int64_t k, int64_t kp, uint8_t *out, int num_sms);
cudaError_t launch_expand_transpose(cudaStream_t st, int fmt, const uint64_t *B, int64_t ldb, int64_t k0, int64_t k,
                                    int64_t n, int64_t kp, uint8_t *out, int num_sms);
cudaError_t launch_parity(cudaStream_t st, const float *D, int64_t ldd, int64_t rows, int64_t n, uint64_t *C,
                          int64_t ldc, int num_sms);
// library GEMM (built only with GF2_WITH_CUBLASLT; otherwise create returns null)
constexpr bool kLibraryGemm =
#ifdef GF2_WITH_CUBLASLT
    true;
#else
    false;
#endif
void *gemm_lt_create();
void gemm_lt_destroy(void *g);
int gemm_counts(void *g, cudaStream_t st, int fmt, const uint8_t *Ax, const uint8_t *Bxt, float *D, int64_t rows,
                int64_t n, int64_t kp, int64_t ldd);
// blocked PLE (kernels_blocked.cu)
cudaError_t launch_gather_lbits(cudaStream_t st, const uint64_t *A, int64_t ld, int64_t W, int64_t row0, int64_t rows,
                                int64_t c0, int64_t kb, int64_t kw, uint64_t *out, int num_sms);
cudaError_t launch_gather_pivbits(cudaStream_t st, const uint64_t *A, int64_t ld, int64_t W, int64_t row0,
                                  int64_t rows, const int64_t *Qb, int64_t kb, int64_t kw, uint64_t *out,
                                  int num_sms);
// The row moves of the stripes [s0, s1) (their first row r0) on the words
// [w_lo, W): composed into one permutation and applied by a gather and a
// scatter through `scratch` when it holds permute_scratch_bytes (0: the
// block is too wide to compose), else replayed stripe by stripe.
size_t permute_scratch_bytes(int s0, int s1, int64_t m, int64_t r0, int64_t w_lo, int64_t W);
cudaError_t launch_permute_trailing(cudaStream_t st, uint64_t *A, int64_t ld, const StripeDesc *descs, int s0,
                                    int s1, int64_t w_lo, int64_t W, int64_t m, int64_t r0, char *scratch,
                                    size_t scratch_bytes, int num_sms);
cudaError_t setup_blocked_kernels();   // shared-memory limits of the TRSM leaf and the move composition
// fused TRSM leaf (kb <= TRSM_LEAF_MAX): indices into Lp (kb * ceil(kb / 64)
// words), then one launch over the words [w_lo, W)
cudaError_t launch_trsm_leaf(cudaStream_t st, uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *Lt,
                             int64_t ldt, uint64_t *Lp, int64_t w_lo, int64_t W);
constexpr int64_t TRSM_LEAF_MAX = 4096;        // rows of the largest fused leaf
// fused RREF leaf: the back-substitution of the kb <= RREF_LEAF_MAX pivot
// rows A[row0 .. row0 + kb) (pivot columns Qb, their bits on those columns
// gathered in Xb, kw words per row) over the words [w_lo, w_hi); prep = false
// reuses the indices Lp (kb * ceil(kb / 64) words) of an earlier call on the
// same rows
constexpr int64_t RREF_LEAF_MAX = 8192;
cudaError_t launch_rref_leaf(cudaStream_t st, uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *Xb,
                             int64_t kw, const int64_t *Qb, uint64_t *Lp, int64_t w_lo, int64_t w_hi, bool prep);
cudaError_t launch_wait_selftest(cudaStream_t st, int32_t *err, unsigned long long limit_ns);
cudaError_t launch_m4ri_prep(cudaStream_t st, const uint64_t *A, int64_t ld, int64_t W, int s,
                             const StripeDesc *descs, const int32_t *map, uint64_t *S, int64_t ldS, uint64_t *G,
                             uint64_t *IDX, int64_t m, int num_sms);
cudaError_t launch_solve_status(cudaStream_t st, const int64_t *r_dev, const int32_t *flag, int64_t n,
                                int32_t *status);
cudaError_t launch_batched(cudaStream_t st, const gf2_batch_item *items, const int32_t *order, int count,
                           int32_t *next, uint64_t *scratch, int64_t max_rows, int64_t ldS, int grid,
                           BatchTune tune);
cudaError_t launch_batch_fill(cudaStream_t st, const gf2_batch_item *items, int count, uint64_t seed,
                              int num_sms);
size_t batched_scratch_words(int64_t max_rows, int64_t ldS, int grid);
size_t batched_smem_bytes();
int batched_grid(int num_sms);
cudaError_t launch_solve_check(cudaStream_t st, const uint64_t *Aug, int64_t ldaug, int64_t n,
                               int64_t wa, int64_t wb, const int64_t *r_dev, int32_t *flag);
cudaError_t launch_solve_finish(cudaStream_t st, const uint64_t *Aug, int64_t ldaug, int64_t n,
                                int64_t wa, int64_t wb, const int64_t *r_dev, const int64_t *Q,
                                uint64_t *B, int64_t ldb);

}  // namespace gf2
