/*
 * gf2.h -- C ABI of libgf2: dense linear algebra over GF(2) on one GB300 GPU.
 *
 * Method: block-iterative PLE decomposition (Albrecht, Bard & Pernet,
 * "Efficient Dense Gaussian Elimination over the Finite Field with Two
 * Elements", Section 3.2, Algorithm 2), its lazy panel elimination
 * (Algorithm 1), the tabulated trailing update (Algorithms 5-6, "Method of
 * the Four Russians" tables), and the RREF recovered from the PLE form
 * (Section 5).
 *
 * Matrix layout (all entry points): row-major, bit-packed.  A matrix with m
 * rows and n columns occupies m rows of ld_words uint64 words,
 * ld_words >= ceil(n/64).  Column j of a row is bit (j % 64) of word j / 64
 * (least significant bit = lowest column).  Bits at columns >= n (padding)
 * must be zero on input and are zero on output.  A row start that is 16-byte
 * aligned (ld_words even and base 16-byte aligned) takes the vectorised path.
 *
 * Pointers: unless stated otherwise, matrix and vector pointers are DEVICE
 * pointers on the handle's device; scalar outputs (rank, status) are HOST
 * pointers.  The caller owns every buffer; the handle owns its workspace.
 *
 * Asynchrony: work is enqueued on the handle's stream (gf2_set_stream; the
 * default stream otherwise).  Entry points that return a host scalar (rank,
 * solve status) synchronise that stream before returning; the _async forms
 * write the scalar to device memory instead and do not synchronise at the
 * end.  Two options make the host wait inside a call: the blocked PLE
 * (GF2_OPT_PLE_BLOCK, from 65536 pivot columns) reads the rank once per
 * block, and the compact RREF recovery (GF2_OPT_RREF_COMPACT, from 8192 pivot
 * columns) reads the rank and the pivot columns once.
 *
 * Errors: every call returns GF2_OK (0) or a GF2_E* code; gf2_strerror names
 * it.  Invalid sizes or null pointers give GF2_EINVAL before any work is
 * enqueued.  GF2_ECUDA reports a CUDA runtime error (the stream may then hold
 * partially updated data).  m = 0 or n = 0 is valid and gives rank 0.
 */
#ifndef GF2_H
#define GF2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GF2_OK        0
#define GF2_EINVAL    1  /* bad argument: null pointer, negative size, ld too small */
#define GF2_ENOMEM    2  /* device workspace allocation failed                     */
#define GF2_ECUDA     3  /* CUDA runtime error                                     */
#define GF2_ETIMEOUT  4  /* a bounded device-side wait ran out                     */
#define GF2_EINTERNAL 5  /* internal consistency check failed on the device        */

/* gf2_solve status values */
#define GF2_SOLVE_UNIQUE          0  /* rank n: the unique solution              */
#define GF2_SOLVE_UNDERDETERMINED 1  /* consistent, rank < n, free variables = 0 */
#define GF2_SOLVE_INCONSISTENT    2  /* no solution; B holds no solution         */

typedef struct gf2_handle *gf2_handle_t;

/* Create a handle bound to CUDA device `device` (the current device when -1).
 * The handle caches the SM count and owns a workspace grown on demand. */
int gf2_create(gf2_handle_t *handle, int device);
/* Free the handle and its workspace (synchronises its stream first). */
int gf2_destroy(gf2_handle_t handle);
/* Use `stream` (a cudaStream_t, passed as void*) for all later work. */
int gf2_set_stream(gf2_handle_t handle, void *stream);

/*
 * PLE decomposition, in place (Section 2, Definition "PLE Decomposition";
 * Section 3.2, Algorithm 2 "Ensures": A <- L\E, A = P L E, Q_i = column of
 * the i-th pivot of E).
 *   A      device, m x n, ld_words per row.  Overwritten with the
 *          space-sharing form L\E of Section 1.2: entry (i, j) holds L[i][j]
 *          when i > j (only columns j < rank carry L bits; L's columns >= rank
 *          are the identity) and E[i][j] otherwise.
 *   P      device int64[m]: LAPACK-style swap vector (Section 1.2): at step i
 *          rows i and P[i] were exchanged; P[i] = i for i >= rank.
 *   Q      device int64[min(m, n)]: Q[i] = column of pivot i for i < rank,
 *          -1 after.  Pivot rule: leftmost column with a nonzero among the
 *          remaining rows, then the first such row in the current order
 *          (Algorithm 1), so P, Q, L and E are unique.
 *   rank   host int64*: the rank (this call synchronises the stream).
 */
int gf2_ple(gf2_handle_t handle, uint64_t *A, int64_t m, int64_t n, int64_t ld_words,
            int64_t *P, int64_t *Q, int64_t *rank);
/* As gf2_ple, but the rank goes to DEVICE memory rank_dev and nothing waits
   (except, with a PLE block width in effect, once per block for the rank). */
int gf2_ple_async(gf2_handle_t handle, uint64_t *A, int64_t m, int64_t n, int64_t ld_words,
                  int64_t *P, int64_t *Q, int64_t *rank_dev);

/*
 * Reduced row echelon form, in place (Section 2, Definition "Reduced Row
 * Echelon Form"), computed as in Section 5: PLE first, then the RREF is
 * recovered from E by clearing every pivot column above its pivot (from
 * 8192 pivot columns on, by solving only the non-pivot columns:
 * GF2_OPT_RREF_COMPACT).
 *   A      device, overwritten with RREF(A); rows >= rank are zero.
 *   Q      device int64[min(m, n)]: pivot columns (the column rank profile,
 *          Section 2), -1 past the rank.
 *   rank   host int64* (synchronises the stream).
 */
int gf2_rref(gf2_handle_t handle, uint64_t *A, int64_t m, int64_t n, int64_t ld_words,
             int64_t *Q, int64_t *rank);
int gf2_rref_async(gf2_handle_t handle, uint64_t *A, int64_t m, int64_t n, int64_t ld_words,
                   int64_t *Q, int64_t *rank_dev);

/*
 * RREF by M4RI (Algorithm 8, Appendix A): the reduced row echelon form in one
 * sweep over 64-column stripes.  Per stripe the pivots are found below the
 * current rank with the rule of Algorithm 1 (leftmost column, first row,
 * swaps), the stripe's pivot rows are fully reduced (GaussSubmatrix), and
 * every other row -- above and below -- clears its bits in the pivot columns
 * with one table lookup per 8 columns (MakeTable + AddRowsFromTable).
 * Arguments, layout, ownership and errors as gf2_rref / gf2_rref_async; the
 * result is the same unique RREF (Section 2), and Q[0..rank) the same pivot
 * columns.  The tensor-core and TMA options do not apply to it.
 */
int gf2_rref_m4ri(gf2_handle_t handle, uint64_t *A, int64_t m, int64_t n, int64_t ld_words, int64_t *Q,
                  int64_t *rank);
int gf2_rref_m4ri_async(gf2_handle_t handle, uint64_t *A, int64_t m, int64_t n, int64_t ld_words,
                        int64_t *Q, int64_t *rank_dev);

/*
 * Product over GF(2) (Section 3.2: the trailing update is the M4RM
 * multiplication of Albrecht, Bard & Hart; Algorithms 5-6).
 *   C = A B (accumulate = 0) or C ^= A B (accumulate != 0).
 *   A device m x k (lda words), B device k x n (ldb), C device m x n (ldc).
 *   C must not overlap A or B.  Asynchronous.
 * Inner dimensions below GF2_OPT_MUL_GEMM_MIN_K (default 1024, the measured
 * crossover on GB300: at 16384 x k x 16384 the tables win at k = 512, the
 * GEMM at k = 1024) use the
 * tabulated row combinations, 64 columns of A per pass over C; larger ones
 * the library's own block-scaled FP4 tcgen05 GEMM (TMA-fed, parities taken
 * from tensor memory in its epilogue); GF2_OPT_TC_MUL selects the older
 * tcgen05 kernel that expands the bits in shared memory.  The GEMM path
 * holds the operands expanded to FP4 (half a byte per bit; B^T whole, A in
 * blocks of up to 32768 rows) in the handle's workspace.
 */
int gf2_mul(gf2_handle_t handle, uint64_t *C, int64_t ldc, const uint64_t *A, int64_t lda,
            const uint64_t *B, int64_t ldb, int64_t m, int64_t k, int64_t n, int accumulate);

/*
 * Solve A X = B through the PLE decomposition (Section 1: decompositions as
 * the building block for solving dense systems; the conventions are this
 * library's).  A device n x n (lda) is overwritten with L\E of A; B device
 * n x nrhs (ldb) is overwritten with X when a solution exists: X[Q[p]] from
 * back-substitution on E's pivot columns, X[j] = 0 for non-pivot columns j.
 *   solve_status  host int*: GF2_SOLVE_UNIQUE, GF2_SOLVE_UNDERDETERMINED or
 *                 GF2_SOLVE_INCONSISTENT (B's contents are then unspecified).
 * Synchronises the stream.
 */
int gf2_solve(gf2_handle_t handle, uint64_t *A, int64_t n, int64_t lda, uint64_t *B,
              int64_t nrhs, int64_t ldb, int *solve_status);
/* As gf2_solve, but the status goes to DEVICE memory status_dev (one int32)
 * and nothing waits. */
int gf2_solve_async(gf2_handle_t handle, uint64_t *A, int64_t n, int64_t lda, uint64_t *B,
                    int64_t nrhs, int64_t ldb, int32_t *status_dev);

/*
 * Many independent PLE decompositions (each exactly as gf2_ple).  Matrices
 * of at most 4096 x 4096 run in one persistent launch in which every CTA
 * decomposes whole matrices, claimed largest first from a work counter;
 * larger matrices then run the single-matrix path one after another.
 * descs is a HOST array of count descriptors; A, P, Q and rank in each
 * descriptor are DEVICE pointers (rank: one int64).  Matrices must not
 * overlap.  Asynchronous.
 */
typedef struct gf2_desc {
    uint64_t *A;
    int64_t m, n, ld_words;
    int64_t *P;
    int64_t *Q;
    int64_t *rank;
} gf2_desc;
int gf2_ple_batched(gf2_handle_t handle, const gf2_desc *descs, int64_t count);

/*
 * Tuning of the batched kernel (Algorithms 5 and 6 leave the table width
 * open: the paper takes k near log2 n and four tables, Section 3.2 and the
 * appendix).  Matrices fall into size classes by max(m, n):
 *   class 0: <= 128, 1: <= 256, 2: <= 512, 3: <= 1024, 4: <= 2048, 5: <= 4096.
 * Each class runs one table configuration for its 64-column stripes:
 *   config 0: 8 tables of k = 8 bits, tiles of 2 words (default)
 *   config 1: 8 tables of k = 8 bits, tiles of 1 word
 *   config 2: 16 tables of k = 4 bits, tiles of 1 word
 *   config 3: 16 tables of k = 4 bits, tiles of 2 words
 *   config 4: 16 tables of k = 4 bits, tiles of 4 words
 * Results never depend on the configuration.
 * gf2_batched_config: set class size_class (-1: every class) to config
 *   (-1: the default).  GF2_EINVAL for an unknown class or config.
 * gf2_batched_get_config: configs (host int[GF2_BATCH_CLASSES]) <- current.
 * gf2_batched_autotune: for each class, times every configuration on one
 *   wave of seeded random matrices of that class (reps timed runs after a
 *   warm-up, 1 <= reps <= 100) on the handle's stream and keeps the fastest.
 *   ms_out (host double[GF2_BATCH_CLASSES * GF2_BATCH_CONFIGS], may be NULL)
 *   receives the best time of each (class, config).  Synchronous; allocates
 *   and frees up to about 1 GiB of device memory while it runs.
 */
#define GF2_BATCH_CLASSES 6
#define GF2_BATCH_CONFIGS 5
int gf2_batched_config(gf2_handle_t handle, int size_class, int config);
int gf2_batched_get_config(gf2_handle_t handle, int *configs);
int gf2_batched_autotune(gf2_handle_t handle, int reps, double *ms_out);

/*
 * A batched PLE captured once as a CUDA graph and replayed: for callers that
 * run the same batch layout again and again (the matrices' contents change,
 * their addresses and shapes do not).  Every matrix must be at most 4096 x
 * 4096 (larger ones, or count == 0, give GF2_EINVAL), so the graph holds
 * exactly the persistent launch of gf2_ple_batched, with the handle's
 * current batched configuration.
 * gf2_batched_plan_create: copies the descriptors into device memory owned by
 *   the plan and captures the launch; the device buffers named by descs must
 *   stay valid for the plan's lifetime.  Synchronous.
 * gf2_batched_plan_launch: replays the graph on stream (a cudaStream_t as
 *   void*; NULL: the handle's stream).  Asynchronous.  Replays of one plan
 *   must not overlap each other.
 * gf2_batched_plan_destroy: waits for the device to finish all work, then
 *   frees the plan.
 */
typedef struct gf2_batched_plan *gf2_batched_plan_t;
int gf2_batched_plan_create(gf2_handle_t handle, const gf2_desc *descs, int64_t count,
                            gf2_batched_plan_t *plan);
int gf2_batched_plan_launch(gf2_batched_plan_t plan, void *stream);
int gf2_batched_plan_destroy(gf2_batched_plan_t plan);

/* Device workspace gf2_ple / gf2_rref need for an m x n matrix, in bytes. */
size_t gf2_workspace_bytes(gf2_handle_t handle, int64_t m, int64_t n);

/*
 * Host-buffer forms for end-to-end use: A (and P, Q) are HOST pointers
 * (pinned memory gives the fastest copies).  Each call copies the input to
 * the device, runs gf2_ple / gf2_rref there and copies the results back,
 * synchronously.  Device buffers are held in the handle's workspace.
 */
int gf2_ple_host(gf2_handle_t handle, uint64_t *A, int64_t m, int64_t n, int64_t ld_words,
                 int64_t *P, int64_t *Q, int64_t *rank);
int gf2_rref_host(gf2_handle_t handle, uint64_t *A, int64_t m, int64_t n, int64_t ld_words,
                  int64_t *Q, int64_t *rank);

/*
 * PLE with no device memory allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- a process
 * that hands all device memory to its own allocator at start-up, or code
 * that must not stall on cudaMalloc / cudaFree -- and it needs no handle
 * (creating one allocates).
 *   A, P, Q, rank  as gf2_ple (A, P, Q device pointers; rank a host int64*).
 *   stream         a cudaStream_t passed as void* (NULL: the default stream);
 *                  it must belong to the current device (GF2_EINVAL if not),
 *                  since the scratch address used is the current device's.
 * Limits: m <= 4096 and n <= 4096; larger sizes return GF2_EINVAL and enqueue
 * nothing.  Scratch: one fixed array of about 0.5 MiB inside the library,
 * held on every GPU that loads the library until the process exits.  The
 * first call on a device (with that device current) looks up the array's
 * device address.  Every call shares the array and re-initialises what must
 * start from a known state; calls whose work overlaps on the GPU race on it.
 * Synchronises the stream before returning (it reads the rank and pivot
 * counts back to the host between launches), so it can never be captured
 * into a CUDA graph: on a stream that is capturing it returns GF2_EINVAL and
 * enqueues nothing.
 */
int gf2_ple_noalloc(uint64_t *A, int64_t m, int64_t n, int64_t ld_words, int64_t *P, int64_t *Q,
                    int64_t *rank, void *stream);

/*
 * Continuous-batching solve server.  Solving dense systems is the use the
 * paper gives the decomposition (Section 1); serving many of them is this
 * library's: a worker thread owns `slots` execution slots (stream, handle,
 * device buffers for systems up to max_n x max_n with up to max_nrhs right-
 * hand sides, all allocated and sized at creation).  Submitted jobs queue in
 * arrival order; the head of the queue is admitted whenever a slot is free
 * and its device footprint fits in hbm_budget_bytes (0: no limit), so jobs
 * that arrive while others run are started at once and overlap them on the
 * device.  Results (status as gf2_solve, timestamps on gf2_server_clock)
 * are collected with gf2_server_poll.
 *   Job buffers A (n x n, lda), B (n x nrhs, ldb) and X (n x nrhs, ldx) are
 *   HOST pointers (pinned memory recommended) owned by the caller, who must
 *   keep them alive and unmodified until the job's result is polled.
 */
typedef struct gf2_server *gf2_server_t;
typedef struct gf2_solve_job {
    uint64_t id;
    const uint64_t *A;
    int64_t n, lda;
    const uint64_t *B;
    int64_t nrhs, ldb;
    uint64_t *X;
    int64_t ldx;
} gf2_solve_job;
typedef struct gf2_solve_result {
    uint64_t id;
    int status;      /* GF2_SOLVE_*, or -1 when error != 0 */
    int error;       /* GF2_OK or a GF2_E* code */
    double t_submit, t_start, t_done;
} gf2_solve_result;
int gf2_server_create(gf2_server_t *server, int device, int slots, int64_t max_n, int64_t max_nrhs,
                      size_t hbm_budget_bytes);
int gf2_server_submit(gf2_server_t server, const gf2_solve_job *job);
/* Move up to max_results finished jobs into out; *count receives how many. */
int gf2_server_poll(gf2_server_t server, gf2_solve_result *out, int max_results, int *count);
/* Wait until every submitted job has finished. */
int gf2_server_drain(gf2_server_t server);
/* The server's clock, in seconds (monotonic). */
double gf2_server_clock(void);
/* Finish every queued job, then stop the worker and free everything. */
int gf2_server_destroy(gf2_server_t server);

/*
 * Execution options of a handle (value 0 = off, 1 = on):
 *   GF2_OPT_LOOKAHEAD  overlap each stripe's pivot search with the previous
 *                      stripe's trailing update on a side stream (default on)
 *   GF2_OPT_TC_MUL     gf2_mul on the library's own tcgen05 kernel: 0/1
 *                      operands expanded to FP8 in shared memory, the counts
 *                      accumulated in tensor memory and reduced mod 2
 *   GF2_OPT_TC_UPDATE  the PLE / RREF trailing updates on the tensor cores
 *                      instead of the Four-Russians tables
 *   GF2_OPT_TMA_UPDATE the table updates move their rows between HBM and
 *                      shared memory by TMA (a producer warp, five stages)
 *                      where the matrix allows it (16-byte aligned base, even
 *                      ld_words, at least 16 words and 256 rows)
 *   GF2_OPT_MUL_GEMM_MIN_K  gf2_mul with an inner dimension k >= value (0:
 *                      never) runs as an exact tensor-core GEMM: the bits
 *                      expanded to FP4 0/1, the library's own tcgen05
 *                      block-scaled FP4 kernel counting in tensor memory and
 *                      XORing each count's parity into C; below it, the
 *                      Four-Russians tables (default 1024)
 *   GF2_OPT_PLE_BLOCK  value > 0 (a multiple of 64): PLE (and everything
 *                      built on it) decomposes value columns at a time with
 *                      the updates inside the block, then applies the
 *                      block's trailing update at once -- the row moves, the
 *                      TRSM U = L11^-1 A12 and the product A22 ^= L21 U
 *                      through gf2_mul (Algorithm 3's A11 += A10 A01 step);
 *                      the host then reads the rank once per block, so the
 *                      _async calls wait for each block's pivot search;
 *                      0: one table update per 64-column stripe; -1
 *                      (default): blocks of 8192 columns from 65536 pivot
 *                      columns on, else 0.  The block's TRSM halves down to
 *                      leaves of GF2_OPT_TRSM_LEAF rows, each solved by one
 *                      fused launch
 *   GF2_OPT_MUL_GEMM_FORMAT  0 (default): the library's own FP4 GEMM;
 *                      4 / 8: a cuBLASLt GEMM on FP4 E2M1 (NVFP4 scales
 *                      1.0) / FP8 E4M3 operands followed by a parity pass,
 *                      only in a library built with GF2_WITH_CUBLASLT=1
 *                      (GF2_EINVAL otherwise); the counts are exact always
 *   GF2_OPT_RREF_BLOCK value > 0 (a multiple of 64): the RREF recovery
 *                      (gf2_rref, gf2_solve) halves the pivot stripes
 *                      recursively down to blocks of value columns: the
 *                      right half is reduced on its own rows, the rows of the
 *                      left half are cleared on its pivot columns by one
 *                      product through gf2_mul, then the left half follows;
 *                      the table passes run only inside the blocks.  0: one
 *                      table pass per stripe over all rows above it; -1
 *                      (default): blocks of 8192 columns from 32768 pivot
 *                      columns on, else 0
 *   GF2_OPT_WIDE_UPDATE the table updates on 16-byte aligned rows take
 *                      128-byte column tiles with nine tables per stripe
 *                      (eight of 7 bits, one of 8 bits; default on); 0: two
 *                      CTAs share each 128-byte line, 64 bytes each, with
 *                      eight 8-bit tables
 *   GF2_OPT_NAIVE_UPDATE the plain baseline (default off): every trailing
 *                      update (PLE stripes, RREF passes, table products) adds
 *                      the selected generator rows one by one, with no
 *                      tables; for measuring what the tables buy
 *   GF2_OPT_PDL        launch the library's kernels with programmatic
 *                      dependent launch: each kernel is scheduled while the
 *                      one before it on the stream still runs and waits on
 *                      the device for its completion, which hides the launch
 *                      latency between the many short dependent kernels
 *                      (default on; 0: plain stream ordering)
 *   GF2_OPT_PLE_RECURSIVE  with a PLE block width in effect: 1 decomposes
 *                      by Algorithm 3's recursion (Section 3.3) -- the columns
 *                      halved until a half is no wider than the block width,
 *                      each left half's row moves, TRSM and product applied
 *                      to its right sibling's columns only -- instead of
 *                      iterating over the blocks left to right, each block's
 *                      trailing update reaching the row end (default 0)
 *   GF2_OPT_TRSM_LEAF  rows of the fused TRSM leaves of the blocked PLE
 *                      (Algorithm 3's TRSM): 1024, 2048 (default) or 4096.
 *                      Larger diagonal blocks are halved, the halves joined
 *                      by the tensor-core GEMM; a leaf solves its rows in
 *                      64-row table steps in one launch
 *   GF2_OPT_RREF_LEAF  the RREF recovery's base blocks (GF2_OPT_RREF_BLOCK,
 *                      automatic 8192 columns) each reduced by one fused
 *                      back-substitution launch: the block's pivot rows
 *                      times the inverse of their unit upper triangular bits
 *                      on their own pivot columns, in 64-row table steps
 *                      (default 1; 0: one table pass per stripe).  The
 *                      plain, tcgen05 and TMA update forms keep the passes
 *   GF2_OPT_RREF_COMPACT  the RREF recovery on the non-pivot columns only
 *                      (default 1): the RREF is U^-1 E with U the pivot
 *                      rows' bits on their pivot columns, the identity there,
 *                      so E's non-pivot columns are gathered into a compact
 *                      matrix, solved by recursive halving (fused leaves,
 *                      products through gf2_mul) and written back beside the
 *                      identity.  Used from 8192 pivot columns on, or with a
 *                      positive GF2_OPT_RREF_BLOCK (then also the leaves'
 *                      row bound, at most 8192); the host reads the rank and
 *                      the pivot columns once, so the _async calls wait for
 *                      the decomposition.  0: the stripe-wise recovery
 * Look-ahead is on by default; the tcgen05 and TMA forms are off (the
 * register-pipelined table update is faster on every measured shape).
 * Results are identical either way; only the speed differs.
 * GF2_EINVAL for an unknown option, a negative value, a format other
 * than 0, 4 or 8, or a leaf size other than 1024, 2048 or 4096.
 */
#define GF2_OPT_LOOKAHEAD       1
#define GF2_OPT_TC_MUL          2
#define GF2_OPT_TC_UPDATE       3
#define GF2_OPT_TMA_UPDATE      4
#define GF2_OPT_MUL_GEMM_MIN_K  5
#define GF2_OPT_PLE_BLOCK       6
#define GF2_OPT_MUL_GEMM_FORMAT 7
#define GF2_OPT_RREF_BLOCK      8
#define GF2_OPT_WIDE_UPDATE     9
#define GF2_OPT_NAIVE_UPDATE    10
#define GF2_OPT_PDL             11
#define GF2_OPT_PLE_RECURSIVE   12
#define GF2_OPT_TRSM_LEAF       13
#define GF2_OPT_RREF_LEAF       14
#define GF2_OPT_RREF_COMPACT    15
int gf2_set_option(gf2_handle_t handle, int option, int64_t value);

/* Counters of the work enqueued since the last reset (host struct). */
typedef struct gf2_stats {
    int64_t kernel_launches;      /* kernels of this library enqueued          */
    int64_t update_launches;      /* trailing-update kernel launches           */
    double  update_ms;            /* summed CUDA-event time of those launches
                                     (only while profiling is on)              */
    double  update_bytes;         /* algorithmic bytes they moved: 16 bytes per
                                     64-bit word read and written              */
    int64_t panel_fallbacks;      /* stripes that needed the block-wide panel  */
    double  panel_ms;             /* summed event time of the other kernels,   */
    double  prep_ms;              /* by kind (only while profiling is on)      */
    double  rref_prep_ms;
    double  other_ms;
    int64_t update_timed_launches;/* update launches timed while profiling     */
    double  rref_pass_ms;         /* fused RREF stripe passes (rref_pass_kernel,
                                     counted apart from the update): event time,
                                     algorithmic bytes, launches, timed launches */
    double  rref_pass_bytes;
    int64_t rref_pass_launches;
    int64_t rref_pass_timed_launches;
    double  gemm_ms;              /* the own FP4 GEMM (gemm_f4_kernel): event time
                                     and 2 m k n of the launches timed while
                                     profiling (levels 1, 2, 4 and 5), all
                                     launches, timed launches, and 2 m k n of
                                     every launch                               */
    double  gemm_flops;
    int64_t gemm_launches;
    int64_t gemm_timed_launches;
    double  gemm_flops_all;
} gf2_stats;
/* Per-launch event timing: 0 off, 1 the update kernel, the RREF
   back-substitution and the GEMM, 2 every kernel, 3 every 7th update launch
   (only those add to update_ms and update_bytes) and the RREF
   back-substitution, 4 every kernel and a timeline (gf2_get_timeline), 5 the
   GEMM launches only.  While profiling is off update_bytes counts every
   update launch.  Other levels are clamped to 0 .. 5. */
int gf2_set_profiling(gf2_handle_t handle, int on);
/* Read the counters (synchronises the stream to finish the event timing). */
int gf2_get_stats(gf2_handle_t handle, gf2_stats *out);
int gf2_reset_stats(gf2_handle_t handle);
/* Profiling level 4: the timed launches since the last reset, in launch
   order, as (kind, start ms, end ms) triples in out (host, 3 * max_records
   doubles); kind 0 update, 1 panel, 2 prep, 3 RREF prep, 4 other, 5 RREF
   back-substitution (fused pass or leaf), 6 GEMM; times from
   CUDA events recorded on each launch's stream, relative to the first one.
   *count = the number of records (more than max_records: the rest are not
   written).  Synchronises the stream. */
int gf2_get_timeline(gf2_handle_t handle, double *out, int64_t max_records, int64_t *count);

/*
 * Tensor-core carriers of a GF(2) product (Section 3.3: the block step of
 * Algorithm 3 is a matrix multiplication; over GF(2) it is an integer
 * product of 0/1 matrices reduced mod 2).  Four carriers run on sm_103a:
 *   GF2_CARRIER_B1   warp-level mma.sync m16n8k256 on 1-bit operands, AND and
 *                    population count into int32 counts;
 *   GF2_CARRIER_FP8  tcgen05.mma kind::f8f6f4 on E4M3 0/1 (M128 N256 K32);
 *   GF2_CARRIER_FP4  tcgen05.mma kind::mxf4 block-scaled, E2M1 0/1 packed two
 *                    per byte, UE8M0 scales 2^0 per 32 elements (M128 N256 K64);
 *   GF2_CARRIER_NVF4 tcgen05.mma kind::mxf4nvf4 with scale_vec::4X, the same
 *                    operands with UE4M3 scales 1.0 per 16 elements.
 * (The integer tensor-core form kind::i8 is not accepted for sm_103a.)
 * Both calls use the current device and its default stream, allocate a few
 * bytes of device memory and synchronise the device.
 *
 * gf2_carrier_check: one product of bit matrices given as DEVICE words.
 *   B1:       a_bits 16 rows x 4 words (256 bits), b_bits 8 columns x 4
 *             words; counts int32[16 x 8], counts[i * 8 + j] = popcount of
 *             (row i AND column j).
 *   FP8, FP4, NVF4: a_bits 128 rows x 1 word, b_bits 256 columns x 1 word; counts
 *             int32[128 x 256], counts[i * 256 + j] = popcount(a[i] & b[j]).
 * gf2_carrier_rate: `iters` instruction steps per warp (B1: four independent
 *   m16n8k256 per step, 8 warps per CTA, 4 CTAs per SM) or per CTA (FP8: two
 *   K32 MMAs, FP4 / NVF4: one K64 MMA per step, one CTA per SM) on all-ones
 *   operands held in registers or shared memory; *macs_per_s = multiply-adds
 *   per second over the whole GPU, *count_out (may be NULL) = one final
 *   count (iters * 256 for B1, iters * 64 otherwise).  GF2_EINVAL when a
 *   count would not stay exact (iters * 256 >= 2^31 for B1, iters * 64 >=
 *   2^24 otherwise); GF2_ETIMEOUT when a bounded wait for the tensor cores
 *   ran out.
 */
#define GF2_CARRIER_B1  1
#define GF2_CARRIER_FP4 4
#define GF2_CARRIER_FP8 8
#define GF2_CARRIER_NVF4 16
int gf2_carrier_check(int carrier, const uint64_t *a_bits, const uint64_t *b_bits, int32_t *counts);
int gf2_carrier_rate(int carrier, int64_t iters, double *macs_per_s, int64_t *count_out);

/*
 * Failure-detection self-test (no counterpart in the paper): runs one kernel
 * whose bounded mbarrier wait -- the wait the tcgen05 and TMA kernels use --
 * can only end by its limit (limit_us microseconds, at most 10^6), exactly as
 * when an asynchronous copy or product never completes.  Returns
 * GF2_ETIMEOUT when the wait expired and was reported (the expected result);
 * the handle stays usable.  GF2_EINVAL for a bad limit.
 */
int gf2_selftest_wait(gf2_handle_t handle, int64_t limit_us);

/* Static name of a status code. */
const char *gf2_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GF2_H */
