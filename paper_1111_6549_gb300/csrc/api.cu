// api.cu -- host orchestration and the C ABI declared in include/gf2.h.
//
// Block-iterative PLE (Section 3.2, Algorithm 2): the host enqueues, per
// 64-column stripe, the panel (pivot search), the prep (L bits and table
// indices) and the trailing update, all on the handle's stream with no host
// synchronisation in between; the running rank lives in device memory, so
// the stripe loop needs no round trip.  RREF recovery (Section 5) walks the
// stripes backwards with the same update kernel.  Solve runs the same PLE on
// the augmented matrix [A | B] with pivots restricted to A's columns.
#include "common.cuh"
#include "gf2.h"

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <functional>
#include <new>
#include <utility>
#include <vector>

namespace gf2 {
thread_local bool g_pdl = false;
// kernels_rref.cu: a join of the compact recovery with at most a few non-pivot
// columns (C1 ^= X C2 over one-word rows) and whether it fits
bool join_narrow_fits(int64_t kwx, int64_t nnp);
cudaError_t launch_join_narrow(cudaStream_t st, uint64_t *C1, const uint64_t *X, int64_t kwx, const uint64_t *C2,
                               int64_t kx, int nnp, int64_t rows, int num_sms);
}  // namespace gf2

using namespace gf2;

struct gf2_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;   // look-ahead panels run here, overlapping the update
    cudaEvent_t ev_fork = nullptr, ev_u1 = nullptr, ev_p = nullptr;
    bool lookahead = true;
    bool tc_mul = false;           // products on the tensor cores
    bool tc_update = false;        // PLE / RREF trailing updates on the tensor cores
    int num_sms = 1;
    char *ws = nullptr;        // stripe records, indices, staged rows, panel scratch
    size_t ws_cap = 0;
    char *io = nullptr;        // host-API device copies, solve's augmented matrix
    size_t io_cap = 0;
    char *bws = nullptr;       // batched kernel: descriptors, order, per-CTA scratch
    size_t bws_cap = 0;
    char *small = nullptr;     // rank, flags, counters
    int64_t launches = 0;
    int64_t upd_launches = 0;
    int profiling = 0;             // 1: time update launches, 2: every launch, 3: every 7th update launch
    int64_t upd_timed = 0;         // update launches timed (and counted in the byte counter)
    std::vector<cudaEvent_t> ev_free;
    struct Pending { cudaEvent_t e0, e1; int kind; };
    std::vector<Pending> ev_pending;
    double kind_ms[7] = {0, 0, 0, 0, 0, 0, 0};   // update, panel, prep, rref prep, other, rref pass, GEMM
    int64_t gemm_launches = 0;     // gemm_f4_kernel launches
    int64_t gemm_timed = 0;        // of those, timed while profiling
    double gemm_flops = 0;         // 2 m k n of the timed launches
    double gemm_flops_all = 0;     // 2 m k n of every launch
    int64_t rpass_launches = 0;    // fused RREF pass launches (rref_pass_kernel)
    int64_t rpass_timed = 0;
    cudaEvent_t tl_ref = nullptr;  // profiling level 4: the timeline's time origin (first timed event)
    std::vector<double> timeline;  // level 4: (kind, start ms, end ms) per timed launch
    BatchTune btune{};             // batched kernel: table configuration per size class
    bool tma = false;              // update rows move by TMA where A allows it (measured slower)
    int64_t gemm_min_k = 1024;     // gf2_mul: inner dimensions from here on go through the GEMM
    int gemm_fmt = 0;              // 0: own tcgen05 FP4 GEMM; library GEMM (if built in): 4 = FP4 E2M1, 8 = FP8 E4M3
    int64_t rref_block = -1;       // RREF recovery: base block width of the recursive form (0: flat, -1: auto)
    bool wide_update = true;       // table updates on aligned rows: 128-byte tiles, nine tables
    bool naive_update = false;     // plain baseline: trailing updates as one-by-one row additions
    bool pdl = true;               // launches with programmatic dependent launch (GF2_OPT_PDL)
    int64_t ple_block = -1;        // PLE column block for the blocked trailing update (0: per stripe, -1: auto)
    bool ple_recursive = false;    // blocked PLE by recursive halving (Algorithm 3) instead of iterated blocks
    int64_t leaf_rows = 2048;      // blocked PLE: rows of the fused TRSM leaves (1024, 2048 or 4096)
    bool rref_leaf = true;         // RREF recovery: one fused back-substitution launch per base block
    char *lbuf = nullptr;          // blocked PLE: the block's gathered L bits
    size_t lbuf_cap = 0;
    char *tbuf = nullptr;          // blocked PLE: indices of the fused TRSM leaf
    size_t tbuf_cap = 0;
    char *pbuf = nullptr;          // blocked PLE: a block's composed row moves and the moved words
    size_t pbuf_cap = 0;
    char *cbuf = nullptr;          // compact RREF recovery: non-pivot column maps and the reduced bits
    size_t cbuf_cap = 0;
    bool rref_compact = true;      // RREF recovery on the non-pivot columns only (pivot columns: identity)
    void *lt = nullptr;            // cuBLASLt state (created on first use)
    char *gbuf = nullptr;          // expanded operands and fp32 counts of the GEMM path
    size_t gbuf_cap = 0;
    TensorMap2D tmap{};            // TMA descriptor of the last updated matrix
    const void *tm_A = nullptr;
    int64_t tm_m = -1, tm_W = -1, tm_ld = -1;
    bool tm_ok = false;
};

// the own tensor-core product (defined with the C entry points below)
extern "C" {
static int mul_own(gf2_handle *h, uint64_t *C, int64_t ldc, const uint64_t *A, int64_t lda, const uint64_t *B,
                   int64_t ldb, int64_t m, int64_t k, int64_t n);
}

namespace {

// layout of the small device block
constexpr size_t SM_RANK = 0;      // int64 running rank
constexpr size_t SM_ERR = 8;       // int32 internal-check flag
constexpr size_t SM_FALLBACK = 12; // int32 block-wide panel count
constexpr size_t SM_BYTES = 16;    // uint64 algorithmic bytes of update launches
constexpr size_t SM_FLAG = 24;     // int32 solve inconsistency flag
constexpr size_t SM_STATUS = 28;   // int32 solve status
constexpr size_t SM_BYTES2 = 32;   // uint64 algorithmic bytes of fused RREF passes
constexpr size_t SM_BYTES_TOTAL = 256;

int64_t *r_dev(gf2_handle *h) { return reinterpret_cast<int64_t *>(h->small + SM_RANK); }
int32_t *err_dev(gf2_handle *h) { return reinterpret_cast<int32_t *>(h->small + SM_ERR); }
int32_t *fb_dev(gf2_handle *h) { return reinterpret_cast<int32_t *>(h->small + SM_FALLBACK); }
unsigned long long *bytes_dev(gf2_handle *h)
{
    return reinterpret_cast<unsigned long long *>(h->small + SM_BYTES);
}
int32_t *flag_dev(gf2_handle *h) { return reinterpret_cast<int32_t *>(h->small + SM_FLAG); }

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
inline int64_t words_for(int64_t n) { return (n + 63) >> 6; }

struct Layout {
    size_t descs, idx, idx2, gb, map, S, G, ptab, gval, glb, gsrc, P, Q, total;
    int64_t ldS;
};

Layout layout_for(int64_t m, int64_t ncols)
{
    Layout L{};
    const int64_t ns = std::max<int64_t>(words_for(ncols), 1);
    const int64_t W = std::max<int64_t>(words_for(ncols), 1);
    const int64_t mm = std::max<int64_t>(m, 1);
    L.ldS = W + (W & 1);
    size_t off = 0;
    L.descs = off; off = align256(off + (size_t)ns * sizeof(StripeDesc));
    L.idx = off;   off = align256(off + (size_t)mm * 8);
    L.idx2 = off;  off = align256(off + (size_t)mm * 8);                // fused RREF: the next pass's index
    L.gb = off;    off = align256(off + 2 * (size_t)KS * L.ldS * 8);    // fused RREF: reduced pivot rows, by parity
    L.map = off;   off = align256(off + (size_t)mm * 8);   // two halves, by stripe parity
    L.S = off;     off = align256(off + (size_t)SMAX * L.ldS * 8);
    L.G = off;     off = align256(off + (size_t)KS * L.ldS * 8);     // M4RI: reduced pivot rows
    L.ptab = off;  off = align256(off + 2 * PREP_TAB_BYTES);           // prep tables, by stripe parity
    L.gval = off;  off = align256(off + (size_t)mm * 8);
    L.glb = off;   off = align256(off + (size_t)mm * 8);
    L.gsrc = off;  off = align256(off + (size_t)mm * 8);   // source offsets, then positions
    L.P = off;     off = align256(off + (size_t)mm * 8);
    L.Q = off;     off = align256(off + (size_t)std::max<int64_t>(std::min(m, ncols), 1) * 8);
    L.total = off;
    return L;
}

// GF2_OPT_PDL for the launches of one call (restored on exit, so nested
// calls keep the outer setting)
struct PdlScope {
    bool prev;
    explicit PdlScope(bool on) : prev(g_pdl) { g_pdl = on; }
    ~PdlScope() { g_pdl = prev; }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int grow(char **buf, size_t *cap, size_t need, cudaStream_t st)
{
    if (*cap >= need) return GF2_OK;
    if (*buf) {
        cudaStreamSynchronize(st);
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    size_t want = need + need / 4;
    if (cudaMalloc(reinterpret_cast<void **>(buf), want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(reinterpret_cast<void **>(buf), need) != cudaSuccess) {
            cudaGetLastError();
            *buf = nullptr;
            return GF2_ENOMEM;
        }
        want = need;
    }
    *cap = want;
    return GF2_OK;
}

#define CK(expr)                                                  \
    do {                                                          \
        cudaError_t e_ = (expr);                                  \
        if (e_ != cudaSuccess) { cudaGetLastError(); return GF2_ECUDA; } \
    } while (0)

enum { K_UPDATE = 0, K_PANEL = 1, K_PREP = 2, K_RPREP = 3, K_OTHER = 4, K_RPASS = 5, K_GEMM = 6 };

// With profiling on, brackets one launch with a pair of events on the
// handle's stream; the elapsed times are summed per kernel kind later.
struct Timed {
    gf2_handle *h;
    int kind;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr;
    Timed(gf2_handle *h_, int kind_, cudaStream_t st_ = nullptr, bool enable = true)
        : h(h_), kind(kind_), st(st_ ? st_ : h_->stream)
    {
        // level 1: the update, RREF back-substitution and GEMM launches; 2 and
        // 4: every launch; 3: the update and back-substitution launches
        // (updates sampled by the caller); 5: the GEMM launches only
        const int lv = h->profiling;
        const bool on = lv == 2 || lv == 4 ||
                        (lv == 1 && (kind == K_UPDATE || kind == K_RPASS || kind == K_GEMM)) ||
                        (lv == 3 && (kind == K_UPDATE || kind == K_RPASS)) || (lv == 5 && kind == K_GEMM);
        if (!enable || !on) return;
        e0 = take();
        if (e0) cudaEventRecord(e0, st);
    }
    ~Timed()
    {
        if (!e0) return;
        cudaEvent_t e1 = take();
        if (!e1) return;
        cudaEventRecord(e1, st);
        h->ev_pending.push_back({e0, e1, kind});
    }
    cudaEvent_t take()
    {
        cudaEvent_t e = nullptr;
        if (!h->ev_free.empty()) { e = h->ev_free.back(); h->ev_free.pop_back(); }
        else if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); e = nullptr; }
        return e;
    }
};

// Profiling level 3 samples every UPD_SAMPLE-th update launch (odd, so both
// halves of the look-ahead split are sampled): only those are bracketed by
// events and add to the byte counter, which keeps the event overhead out of
// the timed steps while the ratio bytes / time still covers the whole run.
constexpr int64_t UPD_SAMPLE = 7;

int launch_update_counted(gf2_handle *h, const UpdArgs &a_in, cudaStream_t st = nullptr)
{
    if (!st) st = h->stream;
    // the fused RREF passes (their own kernel) are counted and timed apart
    const bool rpass = a_in.rref_fused != 0;
    const int64_t nth = rpass ? h->rpass_launches : h->upd_launches;
    const bool timed = h->profiling != 5 && (h->profiling != 3 || nth % UPD_SAMPLE == 0);
    Timed t(h, rpass ? K_RPASS : K_UPDATE, st, timed);
    UpdArgs a = a_in;
    if (rpass && a.bytes) a.bytes = reinterpret_cast<unsigned long long *>(h->small + SM_BYTES2);
    if (!timed) a.bytes = nullptr;
    else if (h->profiling && t.e0) (rpass ? h->rpass_timed : h->upd_timed) += 1;
    a.err = err_dev(h);
    a.wide = h->wide_update ? 1 : 0;
    a.naive = h->naive_update ? 1 : 0;
    const bool tc = (a.mode == UPD_MUL) ? h->tc_mul : (a.mode == UPD_M4RI ? false : h->tc_update);
    a.tmap = nullptr;
    if (!tc && h->tma && a.mode != UPD_M4RI) {
        const int64_t rows = (a.mode == UPD_MUL) ? a.row_hi : a.m;
        if (a.A != h->tm_A || rows != h->tm_m || a.W != h->tm_W || a.ld != h->tm_ld) {
            h->tm_ok = encode_row_tiles(&h->tmap, a.A, rows, a.W, a.ld);
            h->tm_A = a.A;
            h->tm_m = rows;
            h->tm_W = a.W;
            h->tm_ld = a.ld;
        }
        if (h->tm_ok) a.tmap = &h->tmap;
    }
    if (tc) CK(launch_update_tc(st, a, h->num_sms));
    else CK(launch_update(st, a, h->num_sms));
    h->launches += 1;
    if (rpass) h->rpass_launches += 1;
    else h->upd_launches += 1;
    return GF2_OK;
}

// Enqueue stripes [s_lo, s_hi) of the block-iterative PLE of A (m x ncols,
// pivots among the first npiv columns), updating the words [.., W_upd) of
// every row (the words from W_upd on move with their rows but are otherwise
// left alone).  init: start from rank 0 (P, Q, row map reset).  The rank is
// left in r_dev.
int run_ple_range(gf2_handle *h, uint64_t *A, int64_t m, int64_t ncols, int64_t ld, int64_t npiv, int64_t *P,
                  int64_t *Q, int64_t s_lo, int64_t s_hi, int64_t W_upd, bool init, bool move_rest = true)
{
    const Layout L = layout_for(m, ncols);
    int rc = grow(&h->ws, &h->ws_cap, L.total, h->stream);
    if (rc) return rc;
    char *ws = h->ws;
    StripeDesc *descs = reinterpret_cast<StripeDesc *>(ws + L.descs);
    uint64_t *IDX = reinterpret_cast<uint64_t *>(ws + L.idx);
    int32_t *map = reinterpret_cast<int32_t *>(ws + L.map);
    uint64_t *S = reinterpret_cast<uint64_t *>(ws + L.S);
    PanelScratch gs{reinterpret_cast<uint64_t *>(ws + L.gval), reinterpret_cast<uint64_t *>(ws + L.glb),
                    reinterpret_cast<int32_t *>(ws + L.gsrc),
                    reinterpret_cast<int32_t *>(ws + L.gsrc) + std::max<int64_t>(m, 1)};
    const int64_t qn = std::min(m, npiv);
    const int64_t W = words_for(ncols);
    // The row map has two halves: stripe s uses half s & 1, so the next
    // stripe's panel (running early, on the side stream) never overwrites an
    // entry the current update still reads.
    auto map_of = [&](int64_t s) { return map + (s & 1) * std::max<int64_t>(m, 1); };
    auto ptab_of = [&](int64_t s) {
        return reinterpret_cast<uint64_t *>(ws + L.ptab) + (s & 1) * (3 * PREP_TAB_WORDS);
    };
    if (init) {
        CK(cudaMemsetAsync(map, 0xFF, (size_t)std::max<int64_t>(m, 1) * 8, h->stream));
        {
            Timed t(h, K_OTHER);
            CK(launch_init_ple(h->stream, P, Q, m, qn, nullptr, r_dev(h), h->num_sms));
        }
        h->launches += 1;
    }
    // launches that follow a wait on another stream's event take no PDL
    // attribute, so that the event keeps its full ordering
    // resolve: the previous stripe's update may still be running (its moved
    // rows are read from its staged copies)
    auto panel = [&](cudaStream_t st, int64_t s, bool resolve) -> int {
        PdlScope no_pdl(g_pdl && st == h->stream);
        Timed t(h, K_PANEL, st);
        CK(launch_panel(st, A, m, ld, npiv, (int)s, descs, r_dev(h), P, Q, map_of(s), gs, fb_dev(h),
                        ptab_of(s), resolve ? map_of(s - 1) : nullptr, S, L.ldS));
        h->launches += 1;
        return GF2_OK;
    };
    auto prep = [&](int64_t s, int64_t nw) -> int {
        Timed t(h, K_PREP);
        CK(launch_prep(h->stream, A, m, ld, W, (int)s, descs, map_of(s), S, L.ldS, IDX, err_dev(h),
                       ptab_of(s), h->num_sms, nw));
        h->launches += 1;
        return GF2_OK;
    };
    auto upd = [&](int64_t s, int64_t tp_lo, int64_t tp_hi, int left, int grid, int first_off = 1,
                   cudaStream_t ust = nullptr) -> int {
        UpdArgs a{};
        a.mode = UPD_PLE;
        a.A = A;
        a.ld = ld;
        a.m = m;
        a.W = W_upd;
        a.W_full = move_rest ? W : 0;
        a.desc = descs + s;
        a.stripe = (int)s;
        a.S = S;
        a.ldS = L.ldS;
        a.map = map_of(s);
        a.idx = IDX;
        a.idx_stride = 1;
        a.bytes = bytes_dev(h);
        a.tp_lo = tp_lo;
        a.tp_hi = tp_hi;
        a.left_copies = left;
        a.grid = grid;
        a.first_off = first_off;
        return launch_update_counted(h, a, ust);
    };
    UpdArgs probe{};
    probe.mode = UPD_PLE;
    probe.A = A;
    probe.ld = ld;
    probe.S = S;
    probe.ldS = L.ldS;
    const bool la = h->lookahead && !h->tc_update && !h->naive_update && h->side && s_hi - s_lo > 1 && update_vectorised(probe) &&
                    h->num_sms >= 8;
    if (!la) {
        // one stream, no look-ahead: launched without PDL (an early-launched
        // grid waiting on its predecessor holds shared memory and threads the
        // running one could use; measured on sparse 10000^2 RREF: 38.3 ms with
        // PDL against 24.1 ms without)
        PdlScope no_pdl(false);
        for (int64_t s = s_lo; s < s_hi; ++s) {
            if ((rc = panel(h->stream, s, false))) return rc;
            if ((rc = prep(s, -1))) return rc;
            if ((rc = upd(s, 0, -1, 1, 0))) return rc;
        }
        return GF2_OK;
    }
    // Look-ahead: prep(s) also applies stripe s's update to the next stripe's
    // word of every row, so the panel of stripe s+1 runs right after it on the
    // main stream, reading the rows stripe s moved from their staged copies,
    // while the update of stripe s (from the word after that one, on all but
    // two SMs) runs on the side stream; prep(s+1) waits for both.  The chain
    // prep -> panel -> prep that bounds narrow trailing blocks thus stays on
    // one stream.
    CK(cudaEventRecord(h->ev_fork, h->stream));
    CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    if ((rc = panel(h->stream, s_lo, false))) return rc;
    for (int64_t s = s_lo; s < s_hi; ++s) {
        if (s > s_lo) CK(cudaStreamWaitEvent(h->stream, h->ev_p, 0));   // the update of stripe s - 1
        if (s + 1 < s_hi) {
            {
                PdlScope no_pdl(g_pdl && s == s_lo);       // prep(s > s_lo) follows a wait on the update
                if ((rc = prep(s, s + 1))) return rc;
            }
            CK(cudaEventRecord(h->ev_u1, h->stream));
            CK(cudaStreamWaitEvent(h->side, h->ev_u1, 0));
            {
                PdlScope no_pdl(false);
                if ((rc = upd(s, 0, -1, 1, h->num_sms - 2, 2, h->side))) return rc;
            }
            CK(cudaEventRecord(h->ev_p, h->side));
            if ((rc = panel(h->stream, s + 1, true))) return rc;
        } else {
            {
                PdlScope no_pdl(g_pdl && s == s_lo);
                if ((rc = prep(s, -1))) return rc;
            }
            if ((rc = upd(s, 0, -1, 1, 0))) return rc;
        }
    }
    return GF2_OK;
}

// X <- L^-1 X for the kb rows X = A[row0 .. row0+kb), words [w_lo, W), with
// L the unit lower triangular kb x kb matrix whose strictly lower bits are the
// gathered rows Lt (kb x ldt words, aligned).  Large blocks split in halves
// (X2 ^= L21 X1 through the GEMM between the two half solves); from 1024
// rows down, one fused leaf launch (kernels_blocked.cu: 64-row steps, each CTA
// owning two words of every row) after one launch that forms its indices.
static int trsm_lower(gf2_handle *h, uint64_t *A, int64_t ld, int64_t row0, int64_t kb, const uint64_t *Lt,
                      int64_t ldt, int64_t w_lo, int64_t W, int64_t ncols)
{
    if (kb > h->leaf_rows) {
        const int64_t hh = ((kb / 2) + 63) & ~int64_t(63);
        int rc = trsm_lower(h, A, ld, row0, hh, Lt, ldt, w_lo, W, ncols);
        if (rc) return rc;
        // the product always through the tensor-core GEMM: even at the
        // smallest split (k = 1024) it beats 64-row table passes
        rc = mul_own(h, A + (row0 + hh) * ld + w_lo, ld, Lt + hh * ldt, ldt, A + row0 * ld + w_lo, ld, kb - hh, hh,
                     ncols - 64 * w_lo);
        if (rc) return rc;
        return trsm_lower(h, A, ld, row0 + hh, kb - hh, Lt + hh * ldt + hh / 64, ldt, w_lo, W, ncols);
    }
    const size_t need = (size_t)kb * (size_t)words_for(kb) * 8;
    int rc = grow(&h->tbuf, &h->tbuf_cap, need, h->stream);
    if (rc) return rc;
    {
        Timed t(h, K_OTHER);
        CK(launch_trsm_leaf(h->stream, A, ld, row0, kb, Lt, ldt, reinterpret_cast<uint64_t *>(h->tbuf), w_lo, W));
    }
    h->launches += 2;
    return GF2_OK;
}

// The trailing update of a finished column block: the block's stripes
// [s0, s1) took the pivot rows [r0, r1); the words [w_lo, w_hi) right of it
// (columns up to ncols_hi) get the block's row moves, U = L11^-1 A12 on the
// pivot rows and A22 ^= L21 U below them (Algorithm 3's TRSM and product).
static int block_trailing(gf2_handle *h, uint64_t *A, int64_t m, int64_t ncols, int64_t ld, int64_t s0, int64_t s1,
                          int64_t r0, int64_t r1, int64_t w_lo, int64_t w_hi, int64_t ncols_hi)
{
    const int64_t W = words_for(ncols);
    {
        const size_t pb = permute_scratch_bytes((int)s0, (int)s1, m, r0, w_lo, w_hi);
        if (pb > 0) {
            const int rc = grow(&h->pbuf, &h->pbuf_cap, pb, h->stream);
            if (rc) return rc;
        }
        Timed t(h, K_OTHER);
        CK(launch_permute_trailing(h->stream, A, ld,
                                   reinterpret_cast<StripeDesc *>(h->ws + layout_for(m, ncols).descs), (int)s0,
                                   (int)s1, w_lo, w_hi, m, r0, pb > 0 ? h->pbuf : nullptr, pb > 0 ? h->pbuf_cap : 0,
                                   h->num_sms));
    }
    h->launches += permute_scratch_bytes((int)s0, (int)s1, m, r0, w_lo, w_hi) > 0 ? 4 : 1;
    const int64_t kb = r1 - r0;
    if (kb <= 0 || w_lo >= w_hi) return GF2_OK;
    // the block's L bits, rows r0 .. m, aligned
    const int64_t kw = words_for(kb);
    int rc = grow(&h->lbuf, &h->lbuf_cap, (size_t)(m - r0) * kw * 8, h->stream);
    if (rc) return rc;
    uint64_t *Lt = reinterpret_cast<uint64_t *>(h->lbuf);
    {
        Timed t(h, K_OTHER);
        CK(launch_gather_lbits(h->stream, A, ld, W, r0, m - r0, r0, kb, kw, Lt, h->num_sms));
    }
    h->launches += 1;
    // U = L11^-1 A[r0:r1, w_lo:w_hi)
    if ((rc = trsm_lower(h, A, ld, r0, kb, Lt, kw, w_lo, w_hi, ncols_hi))) return rc;
    // A[r1:m, w_lo:w_hi) ^= L21 U
    if (r1 < m) {
        rc = gf2_mul(h, A + r1 * ld + w_lo, ld, Lt + kb * kw, kw, A + r0 * ld + w_lo, ld, m - r1, kb,
                     ncols_hi - 64 * w_lo, 1);
        if (rc) return rc;
    }
    return GF2_OK;
}

static int read_rank(gf2_handle *h, int64_t *r)
{
    CK(cudaMemcpyAsync(r, r_dev(h), sizeof(*r), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GF2_OK;
}

// Enqueue the PLE of A (m x ncols, pivots among the first npiv columns); the
// rank is left in r_dev.  Three forms:
//  - per stripe (no block width): Algorithm 2's loop over all stripes, each
//    stripe's update over the whole row;
//  - iterated blocks (GF2_OPT_PLE_BLOCK, the default from 65536 pivot
//    columns): the stripes are decomposed block by block with their updates
//    restricted to the block, and the columns right of each block get the
//    block's whole trailing update at once (block_trailing);
//  - recursive (GF2_OPT_PLE_RECURSIVE): Algorithm 3, the columns halved until
//    a half is no wider than the block width, each left half's trailing
//    update applied to its right sibling's columns only.
// The host reads the rank once per block.
int run_ple(gf2_handle *h, uint64_t *A, int64_t m, int64_t ncols, int64_t ld, int64_t npiv, int64_t *P,
            int64_t *Q)
{
    const int64_t W = words_for(ncols), ns = words_for(npiv);
    // stripes per block; automatic: blocks of 8192 columns from 65536 pivot
    // columns on (measured on GB300 with the own GEMM and the fused TRSM
    // leaves: 65536^2 PLE 62.3 ms against 63.6 ms with 16384-column blocks,
    // 62.6 ms with 12288 and 97 ms per stripe; at 32768^2 blocking does not
    // pay)
    const int64_t bs = h->ple_block >= 0 ? h->ple_block / 64 : (npiv >= 65536 ? 128 : 0);
    if (bs <= 0 || ns <= bs) return run_ple_range(h, A, m, ncols, ld, npiv, P, Q, 0, ns, W, true);
    if (h->ple_recursive) {
        // rec(a, b, w_hi): the stripes [a, b), whose updates reach the word
        // w_hi (W at the root; the right sibling's end below it)
        std::function<int(int64_t, int64_t, int64_t)> rec = [&](int64_t a, int64_t b, int64_t w_hi) -> int {
            const bool last = w_hi == W;
            if (b - a <= bs) return run_ple_range(h, A, m, ncols, ld, npiv, P, Q, a, b, w_hi, a == 0, last);
            const int64_t mid = a + (b - a + 1) / 2;
            int64_t r0 = 0, r1 = 0;
            int rc;
            if (a > 0 && (rc = read_rank(h, &r0))) return rc;
            if ((rc = rec(a, mid, mid))) return rc;
            if ((rc = read_rank(h, &r1))) return rc;
            rc = block_trailing(h, A, m, ncols, ld, a, mid, r0, r1, mid, w_hi, std::min(ncols, 64 * w_hi));
            if (rc) return rc;
            return rec(mid, b, w_hi);
        };
        return rec(0, ns, W);
    }
    int64_t r0 = 0;
    for (int64_t s0 = 0; s0 < ns; s0 += bs) {
        const int64_t s1 = std::min(ns, s0 + bs);
        const bool last = s1 == ns;
        const int64_t W_upd = last ? W : s1;
        int rc = run_ple_range(h, A, m, ncols, ld, npiv, P, Q, s0, s1, W_upd, s0 == 0, last);
        if (rc) return rc;
        if (last) break;
        int64_t r1 = 0;
        if ((rc = read_rank(h, &r1))) return rc;
        rc = block_trailing(h, A, m, ncols, ld, s0, s1, r0, r1, W_upd, W, ncols);
        if (rc) return rc;
        r0 = r1;                                         // later blocks still run: their stripe records
    }                                                    // (rank 0 once no row is left) feed the RREF
    return GF2_OK;
}

// The compact RREF recovery (Section 5's RREF from the PLE decomposition):
// with E the decomposed matrix's first r rows (L bits cleared) and
// U = E[:, Q] their unit upper triangular bits on the pivot columns, the RREF
// is U^-1 E.  On the pivot columns that is the identity, so only the
// non-pivot columns are computed: C = E[:, NP] is gathered into a compact
// matrix, C <- U^-1 C by recursive halving of the rows (the lower half
// reduced first, the upper rows then cleared on its pivot columns by one
// product C1 ^= X C2 through gf2_mul, X their bits on those columns),
// with fused back-substitution leaves of at most `leaf` rows, and the rows
// are written back as the identity on Q plus C on NP.  The host reads the
// rank and the pivot columns once.
static int rref_compact(gf2_handle *h, uint64_t *A, int64_t m, int64_t ncols, int64_t ld, const int64_t *Qs,
                        int64_t leaf)
{
    const int64_t W = words_for(ncols);
    int64_t r = 0;
    CK(cudaMemcpyAsync(&r, r_dev(h), sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (r <= 0) return GF2_OK;                           // every row cleared already
    std::vector<int64_t> q((size_t)r);
    CK(cudaMemcpyAsync(q.data(), Qs, (size_t)r * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // the non-pivot columns, and per word their mask and first compact position
    std::vector<int64_t> np;
    np.reserve((size_t)(ncols - r));
    std::vector<uint64_t> npmask((size_t)W, 0ull);
    std::vector<int64_t> npstart((size_t)W, 0);
    {
        size_t j = 0;
        for (int64_t c = 0; c < ncols; ++c) {
            if (j < q.size() && q[j] == c) { ++j; continue; }
            if (npmask[(size_t)(c >> 6)] == 0) npstart[(size_t)(c >> 6)] = (int64_t)np.size();
            npmask[(size_t)(c >> 6)] |= 1ull << (c & 63);
            np.push_back(c);
        }
    }
    const int64_t nnp = (int64_t)np.size();
    const int64_t kwn = std::max<int64_t>(words_for(nnp), 1);
    const size_t off_mask = align256(std::max<size_t>(np.size(), 1) * 8);
    const size_t off_start = off_mask + align256((size_t)W * 8);
    const size_t off_c = off_start + align256((size_t)W * 8);
    int rc = grow(&h->cbuf, &h->cbuf_cap, off_c + (size_t)r * kwn * 8, h->stream);
    if (rc) return rc;
    int64_t *d_np = reinterpret_cast<int64_t *>(h->cbuf);
    uint64_t *d_mask = reinterpret_cast<uint64_t *>(h->cbuf + off_mask);
    int64_t *d_start = reinterpret_cast<int64_t *>(h->cbuf + off_start);
    uint64_t *C = reinterpret_cast<uint64_t *>(h->cbuf + off_c);
    if (nnp > 0) CK(cudaMemcpyAsync(d_np, np.data(), (size_t)nnp * 8, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(d_mask, npmask.data(), (size_t)W * 8, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(d_start, npstart.data(), (size_t)W * 8, cudaMemcpyHostToDevice, h->stream));
    if (nnp > 0) {
        {
            Timed t(h, K_OTHER);
            CK(launch_gather_pivbits(h->stream, A, ld, W, 0, r, d_np, nnp, kwn, C, h->num_sms));
        }
        h->launches += 1;
        std::function<int(int64_t, int64_t)> solve = [&](int64_t ra, int64_t rb) -> int {
            const int64_t kb = rb - ra;
            if (kb <= 0) return GF2_OK;
            if (kb <= leaf) {
                const int64_t kw = words_for(kb);
                int rc2 = grow(&h->lbuf, &h->lbuf_cap, (size_t)kb * kw * 8, h->stream);
                if (rc2) return rc2;
                rc2 = grow(&h->tbuf, &h->tbuf_cap, (size_t)kb * kw * 8, h->stream);
                if (rc2) return rc2;
                uint64_t *Xb = reinterpret_cast<uint64_t *>(h->lbuf);
                {
                    Timed t(h, K_OTHER);
                    CK(launch_gather_pivbits(h->stream, A, ld, W, ra, kb, Qs + ra, kb, kw, Xb, h->num_sms));
                }
                {
                    Timed t(h, K_RPASS);
                    CK(launch_rref_leaf(h->stream, C, kwn, ra, kb, Xb, kw, nullptr,
                                        reinterpret_cast<uint64_t *>(h->tbuf), 0, kwn, true));
                    if (t.e0) h->rpass_timed += 1;
                }
                h->launches += 3;
                h->rpass_launches += 1;
                return GF2_OK;
            }
            const int64_t mid = ra + (((kb / 2) + 63) & ~int64_t(63));
            int rc2 = solve(mid, rb);
            if (rc2) return rc2;
            const int64_t rows = mid - ra, kx = rb - mid, kwx = words_for(kx);
            rc2 = grow(&h->lbuf, &h->lbuf_cap, (size_t)rows * kwx * 8, h->stream);
            if (rc2) return rc2;
            uint64_t *X = reinterpret_cast<uint64_t *>(h->lbuf);
            {
                Timed t(h, K_OTHER);
                CK(launch_gather_pivbits(h->stream, A, ld, W, ra, rows, Qs + mid, kx, kwx, X, h->num_sms));
            }
            h->launches += 1;
            if (kwn == 1 && join_narrow_fits(kwx, nnp)) {
                // at most a few non-pivot columns: parities of X's rows with
                // C2's columns, no operand expansion
                Timed t(h, K_OTHER);
                CK(launch_join_narrow(h->stream, C + ra, X, kwx, C + mid, kx, (int)nnp, rows, h->num_sms));
                h->launches += 1;
            } else {
                rc2 = gf2_mul(h, C + ra * kwn, kwn, X, kwx, C + mid * kwn, kwn, rows, kx, nnp, 1);
            }
            if (rc2) return rc2;
            return solve(ra, mid);
        };
        if ((rc = solve(0, r))) return rc;
    }
    {
        Timed t(h, K_OTHER);
        CK(launch_rref_scatter(h->stream, A, ld, W, r, Qs, C, kwn, d_mask, d_start, h->num_sms));
    }
    h->launches += 1;
    return GF2_OK;
}

// Enqueue the RREF recovery of a matrix that run_ple just decomposed.
int run_rref_back(gf2_handle *h, uint64_t *A, int64_t m, int64_t ncols, int64_t ld, int64_t npiv, const int64_t *Qs)
{
    const Layout L = layout_for(m, ncols);
    StripeDesc *descs = reinterpret_cast<StripeDesc *>(h->ws + L.descs);
    uint64_t *IDX = reinterpret_cast<uint64_t *>(h->ws + L.idx);
    const int64_t W = words_for(ncols);
    const int64_t ns = words_for(npiv);
    {
        Timed t(h, K_OTHER);
        CK(launch_rref_lclear(h->stream, A, m, W, ld, r_dev(h), h->num_sms));
    }
    h->launches += 1;
    // the compact form (default from 8192 pivot columns on, or with an
    // explicit base block width, which then bounds its leaves)
    const bool leaf_ok = h->rref_leaf && !h->naive_update && !h->tc_update && !h->tma;
    if (h->rref_compact && leaf_ok && (h->rref_block > 0 || (h->rref_block < 0 && npiv >= 8192)))
        return rref_compact(h, A, m, ncols, ld, Qs,
                            std::min<int64_t>(h->rref_block > 0 ? h->rref_block : 2048, RREF_LEAF_MAX));
    // one stripe's back-substitution: rows [row_lo, r_s) over the words
    // [c_s, W) except [skip_lo, skip_hi), where those rows and the stripe's
    // pivot rows are known to be zero
    auto stripe = [&](int64_t s, int64_t row_lo, int64_t skip_lo, int64_t skip_hi) -> int {
        const bool split = skip_lo < skip_hi;
        {
            Timed t(h, K_RPREP);
            CK(launch_rref_prep(h->stream, A, ld, split && skip_hi >= W ? skip_lo : W, (int)s, descs, IDX, m,
                                h->num_sms));
        }
        h->launches += 1;
        UpdArgs a{};
        a.tp_lo = 0;
        a.tp_hi = -1;
        a.left_copies = 1;
        a.mode = UPD_RREF;
        a.A = A;
        a.ld = ld;
        a.m = m;
        a.W = split ? skip_lo : W;
        a.row_lo = row_lo;
        a.desc = descs + s;
        a.stripe = (int)s;
        a.idx = IDX;
        a.idx_stride = 1;
        a.bytes = bytes_dev(h);
        // the pipelined table kernel leaves the skipped words out within one
        // launch; the other forms take the two word ranges one after another
        a.skip_lo = 0;
        a.skip_hi = 0;
        if (split && skip_hi < W && update_vectorised(a) && !h->tc_update && !h->tma && !h->naive_update) {
            a.W = W;
            a.skip_lo = skip_lo;
            a.skip_hi = skip_hi;
            return launch_update_counted(h, a);
        }
        int rc = launch_update_counted(h, a);
        if (rc || !split || skip_hi >= W) return rc;
        a.W = W;
        a.w_lo = skip_hi;
        return launch_update_counted(h, a);
    };
    // The passes of stripes [sa, sb) from the last to the first over the rows
    // [row_lo, r_s).  With the wide table kernel each pass is one launch: the
    // kernel forms the stripe's reduced pivot rows itself (UpdArgs::
    // rref_fused), writes them back one pass later and takes the next pass's
    // index; two small launches bracket the block.  Otherwise rref_prep and
    // the update per stripe.
    uint64_t *IDX2 = reinterpret_cast<uint64_t *>(h->ws + L.idx2);
    uint64_t *GB = reinterpret_cast<uint64_t *>(h->ws + L.gb);
    auto idx_of = [&](int64_t s) { return (s & 1) ? IDX2 : IDX; };
    auto gb_of = [&](int64_t s) { return GB + (s & 1) * (int64_t)KS * L.ldS; };
    UpdArgs fprobe{};
    fprobe.mode = UPD_RREF;
    fprobe.A = A;
    fprobe.ld = ld;
    const bool fusable = update_vectorised(fprobe) && h->wide_update && !h->tc_update && !h->tma && !h->naive_update;
    auto passes = [&](int64_t sa, int64_t sb, int64_t row_lo, int64_t skip_lo, int64_t skip_hi) -> int {
        if (!fusable) {
            PdlScope no_pdl(false);                      // as the PLE loop without look-ahead
            for (int64_t s = sb - 1; s >= sa; --s) {
                int rc = stripe(s, row_lo, skip_lo, skip_hi);
                if (rc) return rc;
            }
            return GF2_OK;
        }
        const bool split = skip_lo < skip_hi;
        const int64_t Wp = split && skip_hi >= W ? skip_lo : W;
        const int64_t sk_lo = split && skip_hi < W ? skip_lo : 0, sk_hi = split && skip_hi < W ? skip_hi : 0;
        {
            Timed t(h, K_RPREP);
            CK(launch_rref_aux(h->stream, A, ld, nullptr, nullptr, L.ldS, Wp, sk_lo, sk_hi, descs + (sb - 1),
                               idx_of(sb - 1), row_lo, h->num_sms));
        }
        h->launches += 1;
        for (int64_t s = sb - 1; s >= sa; --s) {
            UpdArgs a{};
            a.tp_lo = 0;
            a.tp_hi = -1;
            a.left_copies = 1;
            a.mode = UPD_RREF;
            a.A = A;
            a.ld = ld;
            a.m = m;
            a.W = Wp;
            a.skip_lo = sk_lo;
            a.skip_hi = sk_hi;
            a.row_lo = row_lo;
            a.desc = descs + s;
            a.stripe = (int)s;
            a.idx = idx_of(s);
            a.idx_stride = 1;
            a.bytes = bytes_dev(h);
            a.rref_fused = 1;
            a.gbuf_w = gb_of(s);
            a.gbuf_r = gb_of(s + 1);
            a.ldg = L.ldS;
            a.flush_desc = s + 1 < sb ? descs + (s + 1) : nullptr;
            a.snap_desc = s > sa ? descs + (s - 1) : nullptr;
            a.idx_next = idx_of(s - 1);
            int rc = launch_update_counted(h, a);
            if (rc) return rc;
        }
        {
            Timed t(h, K_RPREP);
            CK(launch_rref_aux(h->stream, A, ld, descs + sa, gb_of(sa), L.ldS, Wp, sk_lo, sk_hi, nullptr, nullptr,
                               row_lo, h->num_sms));
        }
        h->launches += 1;
        return GF2_OK;
    };
    // Blocked form (recursive halving down to blocks of rref_base stripes).
    // Invariant of a call on the stripes [a, b): their pivot rows [r_a, r_b)
    // are already zero on every pivot column of the stripes >= b.  The call
    // reduces the right half [mid, b) on its own rows, clears the left half's
    // rows [r_a, r_mid) on the right half's pivot columns at once --
    // rows ^= X G, X their bits on those columns, G the reduced right rows,
    // through gf2_mul -- and recurses into the left half.  Table passes and
    // products skip the words from stripe b's first column up to the first
    // column at or after it that is no pivot: zero in every row involved.
    // A base block's own back-substitution is one fused leaf launch
    // (rref_leaf_kernel) where the options allow it: its rows (at most 64 per
    // stripe) are reduced over the block's words and, past the skipped words,
    // over [sk, W); otherwise one table pass per stripe.
    auto leaf_block = [&](int64_t a, int64_t b, int64_t ra, int64_t rb, int64_t sk) -> int {
        const int64_t kb = rb - ra, kw = words_for(kb);
        int rc = grow(&h->lbuf, &h->lbuf_cap, (size_t)kb * kw * 8, h->stream);
        if (rc) return rc;
        rc = grow(&h->tbuf, &h->tbuf_cap, (size_t)kb * kw * 8, h->stream);
        if (rc) return rc;
        uint64_t *Xb = reinterpret_cast<uint64_t *>(h->lbuf);
        uint64_t *Lp = reinterpret_cast<uint64_t *>(h->tbuf);
        {
            Timed t(h, K_OTHER);
            CK(launch_gather_pivbits(h->stream, A, ld, W, ra, kb, Qs + ra, kb, kw, Xb, h->num_sms));
        }
        const int64_t w_end = b < ns ? b : W;
        {
            Timed t(h, K_RPASS);
            CK(launch_rref_leaf(h->stream, A, ld, ra, kb, Xb, kw, Qs + ra, Lp, a, w_end, true));
            if (t.e0) h->rpass_timed += 1;
        }
        h->launches += 3;
        h->rpass_launches += 1;
        if (w_end < W && sk < W) {
            Timed t(h, K_RPASS);
            CK(launch_rref_leaf(h->stream, A, ld, ra, kb, Xb, kw, Qs + ra, Lp, sk, W, false));
            if (t.e0) h->rpass_timed += 1;
            h->launches += 1;
            h->rpass_launches += 1;
        }
        return GF2_OK;
    };
    // automatic: base blocks of 8192 columns from 32768 pivot columns on
    // (measured on GB300: 65536^2 RREF step 105.7 ms against 108.1 ms with
    // 16384-column blocks; 32768^2 faster than the flat recovery)
    const int64_t base = h->rref_block > 0 ? h->rref_block / 64
                                           : (h->rref_block < 0 && npiv >= 32768 ? 128 : 0);
    if (base > 0 && ns > base) {
        int64_t r = 0;
        CK(cudaMemcpyAsync(&r, r_dev(h), sizeof(r), cudaMemcpyDeviceToHost, h->stream));
        std::vector<int64_t> rs((size_t)ns + 1);
        CK(cudaMemcpy2DAsync(rs.data(), sizeof(int64_t), &descs[0].r, sizeof(StripeDesc), sizeof(int64_t),
                             (size_t)ns, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        rs[(size_t)ns] = r;
        std::vector<int64_t> q((size_t)std::max<int64_t>(r, 1));
        if (r > 0) {
            CK(cudaMemcpyAsync(q.data(), Qs, (size_t)r * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
        // first word past stripe b's cleared words: the word of the first
        // column >= 64 b that is no pivot (W when there is none)
        auto skip_end = [&](int64_t b) -> int64_t {
            if (b >= ns) return W;
            int64_t j = rs[(size_t)b], c = 64 * b;
            while (j < r && q[(size_t)j] == c) ++j, ++c;
            return c >= ncols ? W : c >> 6;
        };
        std::function<int(int64_t, int64_t)> rec = [&](int64_t a, int64_t b) -> int {
            const int64_t ra = rs[(size_t)a], rb = rs[(size_t)b];
            if (rb == ra) return GF2_OK;                     // no pivot rows: nothing to reduce
            const int64_t sk = skip_end(b);
            if (b - a <= base) {
                if (leaf_ok && rb - ra <= RREF_LEAF_MAX) return leaf_block(a, b, ra, rb, sk);
                return passes(a, b, ra, b < ns ? b : W, sk);
            }
            const int64_t mid = (a + b + 1) / 2;
            int rc = rec(mid, b);
            if (rc) return rc;
            const int64_t rm = rs[(size_t)mid];
            const int64_t kb = rb - rm, rows = rm - ra;
            if (kb > 0 && rows > 0) {
                const int64_t kw = words_for(kb);
                rc = grow(&h->lbuf, &h->lbuf_cap, (size_t)rows * kw * 8, h->stream);
                if (rc) return rc;
                uint64_t *X = reinterpret_cast<uint64_t *>(h->lbuf);
                {
                    Timed t(h, K_OTHER);
                    CK(launch_gather_pivbits(h->stream, A, ld, W, ra, rows, Qs + rm, kb, kw, X, h->num_sms));
                }
                h->launches += 1;
                // G's words [mid, b) and, past the skipped words, [sk, W)
                const int64_t w_end = b < ns ? b : W;
                const int64_t n1 = std::min(64 * w_end, ncols) - 64 * mid;
                rc = gf2_mul(h, A + ra * ld + mid, ld, X, kw, A + rm * ld + mid, ld, rows, kb, n1, 1);
                if (rc) return rc;
                if (w_end < W && sk < W) {
                    rc = gf2_mul(h, A + ra * ld + sk, ld, X, kw, A + rm * ld + sk, ld, rows, kb, ncols - 64 * sk, 1);
                    if (rc) return rc;
                }
            }
            return rec(a, mid);
        };
        return rec(0, ns);
    }
    return passes(0, ns, 0, W, W);
}

// Enqueue M4RI (Algorithm 8): the RREF in one sweep over the stripes.  Per
// stripe: the panel (pivot search below the rank, as for PLE), the reduced
// pivot rows, staged rows and table indices (m4ri_prep), and the table update
// of every row above and below.  The rank is left in r_dev, Q[0..rank) holds
// the pivot columns.
int run_m4ri(gf2_handle *h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *Q)
{
    const Layout L = layout_for(m, n);
    int rc = grow(&h->ws, &h->ws_cap, L.total, h->stream);
    if (rc) return rc;
    char *ws = h->ws;
    StripeDesc *descs = reinterpret_cast<StripeDesc *>(ws + L.descs);
    uint64_t *IDX = reinterpret_cast<uint64_t *>(ws + L.idx);
    int32_t *map = reinterpret_cast<int32_t *>(ws + L.map);
    uint64_t *S = reinterpret_cast<uint64_t *>(ws + L.S);
    uint64_t *G = reinterpret_cast<uint64_t *>(ws + L.G);
    int64_t *P = reinterpret_cast<int64_t *>(ws + L.P);
    PanelScratch gs{reinterpret_cast<uint64_t *>(ws + L.gval), reinterpret_cast<uint64_t *>(ws + L.glb),
                    reinterpret_cast<int32_t *>(ws + L.gsrc),
                    reinterpret_cast<int32_t *>(ws + L.gsrc) + std::max<int64_t>(m, 1)};
    const int64_t W = words_for(n);
    CK(cudaMemsetAsync(map, 0xFF, (size_t)std::max<int64_t>(m, 1) * 4, h->stream));
    {
        Timed t(h, K_OTHER);
        CK(launch_init_ple(h->stream, P, Q, m, std::min(m, n), nullptr, r_dev(h), h->num_sms));
    }
    h->launches += 1;
    for (int64_t s = 0; s < W; ++s) {
        {
            Timed t(h, K_PANEL);
            CK(launch_panel(h->stream, A, m, ld, n, (int)s, descs, r_dev(h), P, Q, map, gs, fb_dev(h), nullptr));
        }
        {
            Timed t(h, K_PREP);
            CK(launch_m4ri_prep(h->stream, A, ld, W, (int)s, descs, map, S, L.ldS, G, IDX, m, h->num_sms));
        }
        h->launches += 2;
        UpdArgs a{};
        a.mode = UPD_M4RI;
        a.A = A;
        a.ld = ld;
        a.m = m;
        a.W = W;
        a.desc = descs + s;
        a.stripe = (int)s;
        a.S = S;
        a.ldS = L.ldS;
        a.map = map;
        a.idx = IDX;
        a.idx_stride = 1;
        a.B = G;
        a.ldb = L.ldS;
        a.bytes = bytes_dev(h);
        a.tp_lo = 0;
        a.tp_hi = -1;
        a.left_copies = 1;
        if ((rc = launch_update_counted(h, a))) return rc;
    }
    return GF2_OK;
}

int check_args(gf2_handle *h, const void *A, int64_t m, int64_t n, int64_t ld)
{
    if (!h) return GF2_EINVAL;
    if (m < 0 || n < 0) return GF2_EINVAL;
    if (m > 0 && n > 0) {
        if (!A) return GF2_EINVAL;
        if (ld < words_for(n)) return GF2_EINVAL;
    }
    if (m >= (int64_t(1) << 31)) return GF2_EINVAL;   // slot indices are 32-bit
    return GF2_OK;
}

int finish_sync(gf2_handle *h)
{
    CK(cudaStreamSynchronize(h->stream));
    int32_t err = 0;
    CK(cudaMemcpy(&err, err_dev(h), sizeof(err), cudaMemcpyDeviceToHost));
    if (err) {
        int32_t zero = 0;
        cudaMemcpy(err_dev(h), &zero, sizeof(zero), cudaMemcpyHostToDevice);
        return err == GF2_ETIMEOUT ? GF2_ETIMEOUT : GF2_EINTERNAL;
    }
    return GF2_OK;
}

int ple_impl(gf2_handle *h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *P, int64_t *Q)
{
    if (m == 0) return GF2_OK;
    if (n == 0) {
        CK(launch_init_ple(h->stream, P, Q, m, 0, nullptr, r_dev(h),
                           h->num_sms));
        return GF2_OK;
    }
    return run_ple(h, A, m, n, ld, n, P, Q);
}

}  // namespace

// ============================================================================
extern "C" {

int gf2_create(gf2_handle_t *handle, int device)
{
    if (!handle) return GF2_EINVAL;
    *handle = nullptr;
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return GF2_ECUDA;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || dev >= count) { cudaGetLastError(); return GF2_ECUDA; }
    DeviceGuard g(dev);
    gf2_handle *h = new (std::nothrow) gf2_handle();
    if (!h) return GF2_ENOMEM;
    h->device = dev;
    for (int c = 0; c < BATCH_CLASSES; ++c) h->btune.cfg[c] = BATCH_CFG_DEFAULT;
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete h;
        return GF2_ECUDA;
    }
    if (setup_update_kernel() != cudaSuccess || setup_blocked_kernels() != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return GF2_ECUDA;
    }
    if (cudaMalloc(reinterpret_cast<void **>(&h->small), SM_BYTES_TOTAL) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return GF2_ENOMEM;
    }
    cudaMemset(h->small, 0, SM_BYTES_TOTAL);
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_u1, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_p, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        h->lookahead = false;     // the sequential stripe loop needs none of them
    }
    *handle = h;
    return GF2_OK;
}

int gf2_destroy(gf2_handle_t h)
{
    if (!h) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    cudaStreamSynchronize(h->stream);
    for (auto &p : h->ev_pending) { cudaEventDestroy(p.e0); cudaEventDestroy(p.e1); }
    for (auto e : h->ev_free) cudaEventDestroy(e);
    if (h->side) { cudaStreamSynchronize(h->side); cudaStreamDestroy(h->side); }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_u1) cudaEventDestroy(h->ev_u1);
    if (h->ev_p) cudaEventDestroy(h->ev_p);
    cudaFree(h->ws);
    cudaFree(h->io);
    cudaFree(h->bws);
    cudaFree(h->gbuf);
    cudaFree(h->lbuf);
    cudaFree(h->cbuf);
    cudaFree(h->tbuf);
    cudaFree(h->pbuf);
    gemm_lt_destroy(h->lt);
    cudaFree(h->small);
    delete h;
    return GF2_OK;
}

int gf2_set_stream(gf2_handle_t h, void *stream)
{
    if (!h) return GF2_EINVAL;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    return GF2_OK;
}

size_t gf2_workspace_bytes(gf2_handle_t h, int64_t m, int64_t n)
{
    (void)h;
    if (m <= 0 || n <= 0) return 0;
    return layout_for(m, n).total;
}

int gf2_ple_async(gf2_handle_t h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *P,
                  int64_t *Q, int64_t *rank_dev)
{
    int rc = check_args(h, A, m, n, ld);
    if (rc) return rc;
    if (m > 0 && !P) return GF2_EINVAL;
    if (m > 0 && n > 0 && !Q) return GF2_EINVAL;
    if (!rank_dev) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    if (m == 0 || n == 0) {
        if (m > 0) CK(launch_init_ple(h->stream, P, Q, m, 0, nullptr, r_dev(h), h->num_sms));
        else CK(cudaMemsetAsync(r_dev(h), 0, 8, h->stream));
    } else {
        rc = ple_impl(h, A, m, n, ld, P, Q);
        if (rc) return rc;
    }
    CK(launch_copy_rank(h->stream, r_dev(h), rank_dev));
    h->launches += 1;
    return GF2_OK;
}

int gf2_ple(gf2_handle_t h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *P, int64_t *Q,
            int64_t *rank)
{
    int rc = check_args(h, A, m, n, ld);
    if (rc) return rc;
    if (!rank || (m > 0 && !P) || (m > 0 && n > 0 && !Q)) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    *rank = 0;
    if (m == 0) return GF2_OK;
    if (n == 0) {
        CK(launch_init_ple(h->stream, P, Q, m, 0, nullptr, r_dev(h), h->num_sms));
        h->launches += 1;
        return finish_sync(h);
    }
    rc = run_ple(h, A, m, n, ld, n, P, Q);
    if (rc) return rc;
    CK(cudaMemcpyAsync(rank, r_dev(h), sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    return finish_sync(h);
}

static int rref_enqueue(gf2_handle *h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *Q)
{
    const Layout L = layout_for(m, n);
    int rc = grow(&h->ws, &h->ws_cap, L.total, h->stream);
    if (rc) return rc;
    int64_t *P = reinterpret_cast<int64_t *>(h->ws + L.P);
    rc = run_ple(h, A, m, n, ld, n, P, Q);
    if (rc) return rc;
    return run_rref_back(h, A, m, n, ld, n, Q);
}

int gf2_rref(gf2_handle_t h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *Q, int64_t *rank)
{
    int rc = check_args(h, A, m, n, ld);
    if (rc) return rc;
    if (!rank || (m > 0 && n > 0 && !Q)) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    *rank = 0;
    if (m == 0 || n == 0) return GF2_OK;
    rc = rref_enqueue(h, A, m, n, ld, Q);
    if (rc) return rc;
    CK(cudaMemcpyAsync(rank, r_dev(h), sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    return finish_sync(h);
}

int gf2_rref_async(gf2_handle_t h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *Q,
                   int64_t *rank_dev)
{
    int rc = check_args(h, A, m, n, ld);
    if (rc) return rc;
    if (!rank_dev || (m > 0 && n > 0 && !Q)) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    if (m == 0 || n == 0) {
        CK(cudaMemsetAsync(rank_dev, 0, 8, h->stream));
        return GF2_OK;
    }
    rc = rref_enqueue(h, A, m, n, ld, Q);
    if (rc) return rc;
    CK(launch_copy_rank(h->stream, r_dev(h), rank_dev));
    h->launches += 1;
    return GF2_OK;
}

int gf2_rref_m4ri(gf2_handle_t h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *Q, int64_t *rank)
{
    int rc = check_args(h, A, m, n, ld);
    if (rc) return rc;
    if (!rank || (m > 0 && n > 0 && !Q)) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    *rank = 0;
    if (m == 0 || n == 0) return GF2_OK;
    rc = run_m4ri(h, A, m, n, ld, Q);
    if (rc) return rc;
    CK(cudaMemcpyAsync(rank, r_dev(h), sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    return finish_sync(h);
}

int gf2_rref_m4ri_async(gf2_handle_t h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *Q,
                        int64_t *rank_dev)
{
    int rc = check_args(h, A, m, n, ld);
    if (rc) return rc;
    if (!rank_dev || (m > 0 && n > 0 && !Q)) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    if (m == 0 || n == 0) {
        CK(cudaMemsetAsync(rank_dev, 0, 8, h->stream));
        return GF2_OK;
    }
    rc = run_m4ri(h, A, m, n, ld, Q);
    if (rc) return rc;
    CK(launch_copy_rank(h->stream, r_dev(h), rank_dev));
    h->launches += 1;
    return GF2_OK;
}

// C ^= A B through the library GEMM (kernels_gemm.cu): B is expanded once per
// chunk of at most 2^22 rows (fp32 counts stay exact and below 2^23), A and
// the fp32 counts in row blocks of about 1 GiB of counts.  The FP4 GEMM takes
// only sizes that are multiples of 16, so in that format both operands get
// zero rows up to the next multiple of 16 (their counts are never read).
static int mul_gemm(gf2_handle *h, uint64_t *C, int64_t ldc, const uint64_t *A, int64_t lda, const uint64_t *B,
                    int64_t ldb, int64_t m, int64_t k, int64_t n)
{
    if (!h->lt) {
        h->lt = gemm_lt_create();
        if (!h->lt) return GF2_ECUDA;
    }
    constexpr int64_t KCH = int64_t(1) << 22;
    const int64_t ldd = (n + 15) & ~int64_t(15);
    for (int64_t k0 = 0; k0 < k; k0 += KCH) {
        const int64_t kc = std::min(KCH, k - k0);
        const int64_t kp = (kc + 63) & ~int64_t(63);
        int64_t mb = std::max<int64_t>(1, (int64_t(1) << 30) / (ldd * 4));
        mb = std::min(mb, m);
        mb = (mb + 15) & ~int64_t(15);
        const int fmt = h->gemm_fmt;
        const int64_t np = fmt == 4 ? ldd : n;           // operand rows of B^T handed to the GEMM
        const size_t rowb = (size_t)kp * fmt / 8;        // bytes of one expanded row
        const size_t bbytes = align256((size_t)np * rowb), abytes = align256((size_t)mb * rowb),
                     dbytes = align256((size_t)mb * ldd * 4);
        int rc = grow(&h->gbuf, &h->gbuf_cap, bbytes + abytes + dbytes, h->stream);
        if (rc) return rc;
        uint8_t *B8t = reinterpret_cast<uint8_t *>(h->gbuf);
        uint8_t *A8 = reinterpret_cast<uint8_t *>(h->gbuf + bbytes);
        float *D = reinterpret_cast<float *>(h->gbuf + bbytes + abytes);
        {
            Timed t(h, K_OTHER);
            CK(launch_expand_transpose(h->stream, fmt, B + k0 * ldb, ldb, 0, kc, n, kp, B8t, h->num_sms));
        }
        h->launches += 1;
        if (np > n) CK(cudaMemsetAsync(B8t + (size_t)n * rowb, 0, (size_t)(np - n) * rowb, h->stream));
        for (int64_t i0 = 0; i0 < m; i0 += mb) {
            const int64_t rows = std::min(mb, m - i0);
            {
                Timed t(h, K_OTHER);
                CK(launch_expand_rows(h->stream, fmt, A + i0 * lda, lda, rows, k0, k0 + kc, kp, A8, h->num_sms));
            }
            const int64_t rows_p = fmt == 4 ? (rows + 15) & ~int64_t(15) : rows;   // <= mb
            if (rows_p > rows)
                CK(cudaMemsetAsync(A8 + (size_t)rows * rowb, 0, (size_t)(rows_p - rows) * rowb, h->stream));
            {
                Timed t(h, K_OTHER);
                if (gemm_counts(h->lt, h->stream, fmt, A8, B8t, D, rows_p, np, kp, ldd) != 0) return GF2_ECUDA;
            }
            {
                Timed t(h, K_OTHER);
                CK(launch_parity(h->stream, D, ldd, rows, n, C + i0 * ldc, ldc, h->num_sms));
            }
            h->launches += 2;
        }
    }
    return GF2_OK;
}

// C ^= A B through the own FP4 tcgen05 GEMM (kernels_gemm_f4.cu): per chunk
// of at most 2^22 inner bits (the fp32 counts stay exact and below 2^23), B
// is expanded once to B^T in FP4 and A in row blocks of at most 2^15 rows;
// the GEMM's epilogue XORs the parities into C, so no count reaches memory.
// The expanded operands are padded to whole TMA boxes (256 rows of A, 192 of
// B^T, 128 bytes of inner dimension) with zeros.
static int mul_own(gf2_handle *h, uint64_t *C, int64_t ldc, const uint64_t *A, int64_t lda, const uint64_t *B,
                   int64_t ldb, int64_t m, int64_t k, int64_t n)
{
    constexpr int64_t KCH = int64_t(1) << 22;
    constexpr int64_t MB = int64_t(1) << 15;
    for (int64_t k0 = 0; k0 < k; k0 += KCH) {
        const int64_t kc = std::min(KCH, k - k0);
        const int64_t kp = (kc + 255) & ~int64_t(255);
        const size_t rowb = (size_t)kp / 2;
        const int64_t np = std::max<int64_t>(n, 192);
        const int64_t mb = std::min(m, MB);
        const int64_t mbp = std::max<int64_t>(mb, 256);
        const size_t bbytes = align256((size_t)np * rowb), abytes = align256((size_t)mbp * rowb);
        int rc = grow(&h->gbuf, &h->gbuf_cap, bbytes + abytes, h->stream);
        if (rc) return rc;
        uint8_t *B4t = reinterpret_cast<uint8_t *>(h->gbuf);
        uint8_t *A4 = reinterpret_cast<uint8_t *>(h->gbuf + bbytes);
        {
            Timed t(h, K_OTHER);
            CK(launch_expand_transpose(h->stream, 4, B + k0 * ldb, ldb, 0, kc, n, kp, B4t, h->num_sms));
        }
        h->launches += 1;
        if (np > n) CK(cudaMemsetAsync(B4t + (size_t)n * rowb, 0, (size_t)(np - n) * rowb, h->stream));
        for (int64_t i0 = 0; i0 < m; i0 += mb) {
            const int64_t rows = std::min(mb, m - i0);
            {
                Timed t(h, K_OTHER);
                CK(launch_expand_rows(h->stream, 4, A + i0 * lda, lda, rows, k0, k0 + kc, kp, A4, h->num_sms));
            }
            const int64_t rows_p = std::max<int64_t>(rows, 256);
            if (rows_p > rows)
                CK(cudaMemsetAsync(A4 + (size_t)rows * rowb, 0, (size_t)(rows_p - rows) * rowb, h->stream));
            const double flops = 2.0 * (double)rows * (double)kc * (double)n;
            {
                Timed t(h, K_GEMM);
                CK(launch_gemm_f4(h->stream, C + i0 * ldc, ldc, A4, rows_p, B4t, np, rows, n, kp, err_dev(h),
                                  h->num_sms));
                if (t.e0) {
                    h->gemm_timed += 1;
                    h->gemm_flops += flops;
                }
            }
            h->launches += 2;
            h->gemm_launches += 1;
            h->gemm_flops_all += flops;
        }
    }
    return GF2_OK;
}

int gf2_mul(gf2_handle_t h, uint64_t *C, int64_t ldc, const uint64_t *A, int64_t lda, const uint64_t *B,
            int64_t ldb, int64_t m, int64_t k, int64_t n, int accumulate)
{
    if (!h || m < 0 || k < 0 || n < 0) return GF2_EINVAL;
    if (m == 0 || n == 0) return GF2_OK;
    if (!C || ldc < words_for(n)) return GF2_EINVAL;
    if (k > 0 && (!A || !B || lda < words_for(k) || ldb < words_for(n))) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    const int64_t Wc = words_for(n);
    if (!accumulate)
        CK(cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)Wc * 8, (size_t)m, h->stream));
    if (!h->tc_mul && h->gemm_min_k > 0 && k >= h->gemm_min_k)
        return h->gemm_fmt == 0 ? mul_own(h, C, ldc, A, lda, B, ldb, m, k, n)
                                : mul_gemm(h, C, ldc, A, lda, B, ldb, m, k, n);
    if (h->tc_mul && k > 0) {
        // tensor cores, pipelined tcgen05 kernel: the counts of every inner
        // chunk accumulate in tensor memory, so C is read and written once per
        // group of up to 2^22 columns of A (fp32 counts stay exact below 2^24)
        constexpr int64_t KG = int64_t(1) << 22;
        for (int64_t k0 = 0; k0 < k; k0 += KG) {
            Timed t(h, K_OTHER);
            CK(launch_tc_mul(h->stream, C, ldc, A + k0 / 64, lda, B + k0 * ldb, ldb, m, std::min(KG, k - k0), n,
                             err_dev(h), h->num_sms));
            h->launches += 1;
        }
        return GF2_OK;
    }
    for (int64_t kc = 0; kc < words_for(k); ++kc) {
        UpdArgs a{};
        a.tp_lo = 0;
        a.tp_hi = -1;
        a.left_copies = 1;
        a.mode = UPD_MUL;
        a.A = C;
        a.ld = ldc;
        a.m = m;
        a.W = Wc;
        a.idx = A + kc;
        a.idx_stride = lda;
        a.B = B + kc * 64 * ldb;
        a.ldb = ldb;
        a.gen_count = std::min<int64_t>(64, k - 64 * kc);
        a.row_lo = 0;
        a.row_hi = m;
        a.w_lo = 0;
        a.bytes = bytes_dev(h);
        int rc = launch_update_counted(h, a);
        if (rc) return rc;
    }
    return GF2_OK;
}

// Enqueue a solve; the status (GF2_SOLVE_*) is written to device memory.
static int solve_enqueue(gf2_handle *h, uint64_t *A, int64_t n, int64_t lda, uint64_t *B, int64_t nrhs,
                         int64_t ldb, int32_t *status_dev)
{
    const int64_t wa = words_for(n);
    const int64_t wb = std::max<int64_t>(words_for(nrhs), 1);
    int64_t ldaug = wa + wb;
    ldaug += ldaug & 1;
    const int64_t ncols = 64 * (wa + wb);
    const size_t aug_bytes = align256((size_t)n * ldaug * 8);
    int rc = grow(&h->io, &h->io_cap, aug_bytes, h->stream);
    if (rc) return rc;
    const Layout L = layout_for(n, ncols);
    rc = grow(&h->ws, &h->ws_cap, L.total, h->stream);
    if (rc) return rc;
    uint64_t *Aug = reinterpret_cast<uint64_t *>(h->io);
    int64_t *P = reinterpret_cast<int64_t *>(h->ws + L.P);
    int64_t *Q = reinterpret_cast<int64_t *>(h->ws + L.Q);
    CK(cudaMemsetAsync(Aug, 0, (size_t)n * ldaug * 8, h->stream));
    CK(cudaMemcpy2DAsync(Aug, (size_t)ldaug * 8, A, (size_t)lda * 8, (size_t)wa * 8, (size_t)n,
                         cudaMemcpyDeviceToDevice, h->stream));
    if (nrhs > 0)
        CK(cudaMemcpy2DAsync(Aug + wa, (size_t)ldaug * 8, B, (size_t)ldb * 8, (size_t)words_for(nrhs) * 8,
                             (size_t)n, cudaMemcpyDeviceToDevice, h->stream));
    rc = run_ple(h, Aug, n, ncols, ldaug, n, P, Q);
    if (rc) return rc;
    CK(cudaMemcpy2DAsync(A, (size_t)lda * 8, Aug, (size_t)ldaug * 8, (size_t)wa * 8, (size_t)n,
                         cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemsetAsync(flag_dev(h), 0, 4, h->stream));
    CK(launch_solve_check(h->stream, Aug, ldaug, n, wa, wb, r_dev(h), flag_dev(h)));
    h->launches += 1;
    rc = run_rref_back(h, Aug, n, ncols, ldaug, n, Q);
    if (rc) return rc;
    if (nrhs > 0) {
        CK(launch_solve_finish(h->stream, Aug, ldaug, n, wa, words_for(nrhs), r_dev(h), Q, B, ldb));
        h->launches += 2;
    }
    CK(launch_solve_status(h->stream, r_dev(h), flag_dev(h), n, status_dev));
    h->launches += 1;
    return GF2_OK;
}

int gf2_solve_async(gf2_handle_t h, uint64_t *A, int64_t n, int64_t lda, uint64_t *B, int64_t nrhs,
                    int64_t ldb, int32_t *status_dev)
{
    int rc = check_args(h, A, n, n, lda);
    if (rc) return rc;
    if (!status_dev || nrhs < 0) return GF2_EINVAL;
    if (n > 0 && nrhs > 0 && (!B || ldb < words_for(nrhs))) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    if (n == 0) {
        CK(cudaMemsetAsync(status_dev, 0, sizeof(int32_t), h->stream));
        return GF2_OK;
    }
    return solve_enqueue(h, A, n, lda, B, nrhs, ldb, status_dev);
}

int gf2_solve(gf2_handle_t h, uint64_t *A, int64_t n, int64_t lda, uint64_t *B, int64_t nrhs, int64_t ldb,
              int *solve_status)
{
    int rc = check_args(h, A, n, n, lda);
    if (rc) return rc;
    if (!solve_status || nrhs < 0) return GF2_EINVAL;
    if (n > 0 && nrhs > 0 && (!B || ldb < words_for(nrhs))) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    *solve_status = GF2_SOLVE_UNIQUE;
    if (n == 0) return GF2_OK;
    int32_t *status_dev = reinterpret_cast<int32_t *>(h->small + SM_STATUS);
    rc = solve_enqueue(h, A, n, lda, B, nrhs, ldb, status_dev);
    if (rc) return rc;
    int32_t st = 0;
    CK(cudaMemcpyAsync(&st, status_dev, 4, cudaMemcpyDeviceToHost, h->stream));
    rc = finish_sync(h);
    if (rc) return rc;
    *solve_status = st;
    return GF2_OK;
}

static_assert(sizeof(gf2_desc) == sizeof(gf2_batch_item), "gf2_desc and gf2_batch_item must match");

namespace {

// Matrices up to BATCH_MAX_ROWS x BATCH_MAX_COLS go to the persistent batched
// kernel, largest first; bigger ones take the single-matrix path.
struct BatchSplit {
    std::vector<int32_t> small;
    std::vector<int64_t> large;
    int64_t max_rows = 1, max_w = 1;
};

BatchSplit split_batch(const gf2_desc *descs, int64_t count)
{
    BatchSplit b;
    for (int64_t i = 0; i < count; ++i) {
        const gf2_desc &d = descs[i];
        if (d.m <= BATCH_MAX_ROWS && d.n <= BATCH_MAX_COLS) {
            b.small.push_back((int32_t)i);
            b.max_rows = std::max(b.max_rows, d.m);
            b.max_w = std::max(b.max_w, words_for(d.n));
        } else {
            b.large.push_back(i);
        }
    }
    std::stable_sort(b.small.begin(), b.small.end(), [&](int32_t x, int32_t y) {
        return descs[x].m * descs[x].n > descs[y].m * descs[y].n;
    });
    return b;
}

// Device buffer of one batched launch: descriptors, order, work counter,
// per-CTA scratch.
struct BatchBuf {
    size_t items, order, next, scratch, total;
    int64_t ldS;
    int grid;
};

BatchBuf batch_buf(int num_sms, int64_t count, const BatchSplit &b)
{
    BatchBuf L{};
    L.ldS = b.max_w + (b.max_w & 1);
    L.grid = (int)std::min<int64_t>(batched_grid(num_sms), (int64_t)std::max<size_t>(b.small.size(), 1));
    L.items = 0;
    L.order = align256((size_t)count * sizeof(gf2_desc));
    L.next = L.order + align256(std::max<size_t>(b.small.size(), 1) * sizeof(int32_t));
    L.scratch = L.next + 256;
    L.total = L.scratch + align256(batched_scratch_words(b.max_rows, L.ldS, L.grid) * 8);
    return L;
}

int check_batch(gf2_handle *h, const gf2_desc *descs, int64_t count)
{
    if (!h || count < 0 || (count > 0 && !descs)) return GF2_EINVAL;
    if (count > INT32_MAX / 2) return GF2_EINVAL;
    for (int64_t b = 0; b < count; ++b) {
        const gf2_desc &d = descs[b];
        int rc = check_args(h, d.A, d.m, d.n, d.ld_words);
        if (rc) return rc;
        if (!d.rank || (d.m > 0 && !d.P) || (d.m > 0 && d.n > 0 && !d.Q)) return GF2_EINVAL;
    }
    return GF2_OK;
}

// Enqueue the persistent kernel over the small matrices of a batch whose
// descriptors and order already sit in buf.
int enqueue_batched(gf2_handle *h, cudaStream_t st, char *buf, const BatchBuf &L, const BatchSplit &b,
                    const BatchTune &tune)
{
    auto *items = reinterpret_cast<gf2_batch_item *>(buf + L.items);
    auto *order = reinterpret_cast<int32_t *>(buf + L.order);
    auto *next = reinterpret_cast<int32_t *>(buf + L.next);
    auto *scratch = reinterpret_cast<uint64_t *>(buf + L.scratch);
    CK(cudaMemsetAsync(next, 0, sizeof(int32_t), st));
    CK(launch_batched(st, items, order, (int)b.small.size(), next, scratch, b.max_rows, L.ldS, L.grid, tune));
    h->launches += 1;
    return GF2_OK;
}

}  // namespace

int gf2_ple_batched(gf2_handle_t h, const gf2_desc *descs, int64_t count)
{
    int rc = check_batch(h, descs, count);
    if (rc) return rc;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    const BatchSplit b = split_batch(descs, count);
    if (!b.small.empty()) {
        const BatchBuf L = batch_buf(h->num_sms, count, b);
        rc = grow(&h->bws, &h->bws_cap, L.total, h->stream);
        if (rc) return rc;
        CK(cudaMemcpyAsync(h->bws + L.items, descs, (size_t)count * sizeof(gf2_desc), cudaMemcpyHostToDevice,
                           h->stream));
        CK(cudaMemcpyAsync(h->bws + L.order, b.small.data(), b.small.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, h->stream));
        rc = enqueue_batched(h, h->stream, h->bws, L, b, h->btune);
        if (rc) return rc;
    }
    for (int64_t i : b.large) {
        const gf2_desc &d = descs[i];
        rc = gf2_ple_async(h, d.A, d.m, d.n, d.ld_words, d.P, d.Q, d.rank);
        if (rc) return rc;
    }
    return GF2_OK;
}

static_assert(GF2_BATCH_CLASSES == BATCH_CLASSES && GF2_BATCH_CONFIGS == BATCH_CONFIGS, "batched tuning sizes");

int gf2_batched_config(gf2_handle_t h, int size_class, int config)
{
    if (!h || size_class < -1 || size_class >= BATCH_CLASSES || config < -1 || config >= BATCH_CONFIGS)
        return GF2_EINVAL;
    const int8_t v = (int8_t)(config < 0 ? BATCH_CFG_DEFAULT : config);
    if (size_class < 0)
        for (int c = 0; c < BATCH_CLASSES; ++c) h->btune.cfg[c] = v;
    else
        h->btune.cfg[size_class] = v;
    return GF2_OK;
}

int gf2_batched_get_config(gf2_handle_t h, int *configs)
{
    if (!h || !configs) return GF2_EINVAL;
    for (int c = 0; c < BATCH_CLASSES; ++c) configs[c] = h->btune.cfg[c];
    return GF2_OK;
}

int gf2_batched_autotune(gf2_handle_t h, int reps, double *ms_out)
{
    if (!h || reps < 1 || reps > 100) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    int rc = finish_sync(h);
    if (rc) return rc;
    const int grid = batched_grid(h->num_sms);
    uint64_t state = 0x243F6A8885A308D3ull;
    auto next_u = [&](int64_t lo, int64_t hi) {      // splitmix64, uniform in [lo, hi]
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return lo + (int64_t)(z % (uint64_t)(hi - lo + 1));
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return GF2_ECUDA;
    }
    for (int c = 0; c < BATCH_CLASSES && !rc; ++c) {
        // one wave of matrices of this class, at most 512 MiB of them
        const int64_t hi = int64_t(128) << c, lo = (c == 0) ? 64 : hi / 2 + 1;
        std::vector<gf2_desc> descs;
        size_t words = 0;
        while ((int)descs.size() < grid && words * 8 < (size_t(512) << 20)) {
            gf2_desc d{};
            d.m = next_u(lo, hi);
            d.n = next_u(lo, hi);
            d.ld_words = words_for(d.n);
            d.A = reinterpret_cast<uint64_t *>(words);          // offset for now
            words += (size_t)d.m * d.ld_words;
            descs.push_back(d);
        }
        const int64_t count = (int64_t)descs.size();
        const size_t abytes = align256(words * 8);
        const size_t pbytes = align256((size_t)count * (size_t)hi * 8);
        char *tbuf = nullptr;
        if (cudaMalloc(reinterpret_cast<void **>(&tbuf), 2 * abytes + 2 * pbytes + align256((size_t)count * 8)) !=
            cudaSuccess) {
            cudaGetLastError();
            rc = GF2_ENOMEM;
            break;
        }
        uint64_t *work = reinterpret_cast<uint64_t *>(tbuf), *pristine = reinterpret_cast<uint64_t *>(tbuf + abytes);
        int64_t *P = reinterpret_cast<int64_t *>(tbuf + 2 * abytes);
        int64_t *Q = reinterpret_cast<int64_t *>(tbuf + 2 * abytes + pbytes);
        int64_t *R = reinterpret_cast<int64_t *>(tbuf + 2 * abytes + 2 * pbytes);
        std::vector<gf2_desc> fill = descs;
        for (int64_t i = 0; i < count; ++i) {
            const size_t off = reinterpret_cast<size_t>(descs[i].A);
            descs[i].A = work + off;
            fill[i].A = pristine + off;
            descs[i].P = fill[i].P = P + i * hi;
            descs[i].Q = fill[i].Q = Q + i * hi;
            descs[i].rank = fill[i].rank = R + i;
        }
        const BatchSplit b = split_batch(descs.data(), count);
        const BatchBuf L = batch_buf(h->num_sms, count, b);
        rc = grow(&h->bws, &h->bws_cap, L.total, h->stream);
        if (!rc && (cudaMemcpyAsync(h->bws + L.items, fill.data(), (size_t)count * sizeof(gf2_desc),
                                    cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
                    launch_batch_fill(h->stream, reinterpret_cast<gf2_batch_item *>(h->bws + L.items), (int)count,
                                      0x9E3779B97F4A7C15ull * (c + 1), h->num_sms) != cudaSuccess ||
                    cudaMemcpyAsync(h->bws + L.items, descs.data(), (size_t)count * sizeof(gf2_desc),
                                    cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
                    cudaMemcpyAsync(h->bws + L.order, b.small.data(), b.small.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, h->stream) != cudaSuccess)) {
            cudaGetLastError();
            rc = GF2_ECUDA;
        }
        double best = 1e30;
        int best_cfg = BATCH_CFG_DEFAULT;
        for (int cfg = 0; cfg < BATCH_CONFIGS && !rc; ++cfg) {
            BatchTune t = h->btune;
            t.cfg[c] = (int8_t)cfg;
            double tmin = 1e30;
            for (int k = 0; k <= reps && !rc; ++k) {      // the first run is a warm-up
                float ms = 0.f;
                if (cudaMemcpyAsync(work, pristine, words * 8, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
                    cudaEventRecord(e0, h->stream) != cudaSuccess) {
                    cudaGetLastError();
                    rc = GF2_ECUDA;
                    break;
                }
                rc = enqueue_batched(h, h->stream, h->bws, L, b, t);
                if (rc) break;
                if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    cudaGetLastError();
                    rc = GF2_ECUDA;
                    break;
                }
                if (k > 0) tmin = std::min(tmin, (double)ms);
            }
            if (ms_out) ms_out[c * BATCH_CONFIGS + cfg] = tmin;
            if (tmin < best) { best = tmin; best_cfg = cfg; }
        }
        if (!rc) h->btune.cfg[c] = (int8_t)best_cfg;
        cudaStreamSynchronize(h->stream);
        cudaFree(tbuf);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!rc) rc = finish_sync(h);
    return rc;
}

struct gf2_batched_plan {
    gf2_handle *h = nullptr;
    char *buf = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

int gf2_batched_plan_create(gf2_handle_t h, const gf2_desc *descs, int64_t count, gf2_batched_plan_t *plan)
{
    if (!plan) return GF2_EINVAL;
    *plan = nullptr;
    int rc = check_batch(h, descs, count);
    if (rc) return rc;
    if (count == 0) return GF2_EINVAL;
    const BatchSplit b = split_batch(descs, count);
    if (!b.large.empty()) return GF2_EINVAL;       // plans hold only the persistent launch
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    gf2_batched_plan *p = new (std::nothrow) gf2_batched_plan();
    if (!p) return GF2_ENOMEM;
    p->h = h;
    const BatchBuf L = batch_buf(h->num_sms, count, b);
    auto fail = [&](int code) {
        cudaGetLastError();
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        if (p->cap) cudaStreamDestroy(p->cap);
        cudaFree(p->buf);
        delete p;
        return code;
    };
    if (cudaMalloc(reinterpret_cast<void **>(&p->buf), L.total) != cudaSuccess) return fail(GF2_ENOMEM);
    if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(GF2_ECUDA);
    if (cudaMemcpyAsync(p->buf + L.items, descs, (size_t)count * sizeof(gf2_desc), cudaMemcpyHostToDevice,
                        p->cap) != cudaSuccess ||
        cudaMemcpyAsync(p->buf + L.order, b.small.data(), b.small.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                        p->cap) != cudaSuccess ||
        cudaStreamSynchronize(p->cap) != cudaSuccess)
        return fail(GF2_ECUDA);
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(GF2_ECUDA);
    const int64_t launches = h->launches;
    rc = enqueue_batched(h, p->cap, p->buf, L, b, h->btune);
    h->launches = launches;                         // counted when the graph runs
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->cap, &graph);
    p->graph = graph;
    if (rc || ec != cudaSuccess) return fail(rc ? rc : GF2_ECUDA);
    if (cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) return fail(GF2_ECUDA);
    *plan = p;
    return GF2_OK;
}

int gf2_batched_plan_launch(gf2_batched_plan_t p, void *stream)
{
    if (!p) return GF2_EINVAL;
    DeviceGuard g(p->h->device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : p->h->stream;
    CK(cudaGraphLaunch(p->exec, st));
    p->h->launches += 1;
    return GF2_OK;
}

int gf2_batched_plan_destroy(gf2_batched_plan_t p)
{
    if (!p) return GF2_EINVAL;
    DeviceGuard g(p->h->device);
    cudaDeviceSynchronize();                        // no replay may still use the buffer
    cudaGraphExecDestroy(p->exec);
    cudaGraphDestroy(p->graph);
    cudaStreamDestroy(p->cap);
    cudaFree(p->buf);
    delete p;
    return GF2_OK;
}

int gf2_ple_host(gf2_handle_t h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *P, int64_t *Q,
                 int64_t *rank)
{
    int rc = check_args(h, A, m, n, ld);
    if (rc) return rc;
    if (!rank || (m > 0 && !P) || (m > 0 && n > 0 && !Q)) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    *rank = 0;
    if (m == 0) return GF2_OK;
    const int64_t qn = std::min(m, n);
    const size_t abytes = align256((size_t)m * ld * 8);
    const size_t pbytes = align256((size_t)m * 8);
    const size_t need = abytes + pbytes + align256((size_t)std::max<int64_t>(qn, 1) * 8);
    rc = grow(&h->io, &h->io_cap, need, h->stream);
    if (rc) return rc;
    uint64_t *dA = reinterpret_cast<uint64_t *>(h->io);
    int64_t *dP = reinterpret_cast<int64_t *>(h->io + abytes);
    int64_t *dQ = reinterpret_cast<int64_t *>(h->io + abytes + pbytes);
    if (n > 0) CK(cudaMemcpyAsync(dA, A, (size_t)m * ld * 8, cudaMemcpyHostToDevice, h->stream));
    if (n == 0) {
        CK(launch_init_ple(h->stream, dP, dQ, m, 0, nullptr, r_dev(h), h->num_sms));
    } else {
        rc = run_ple(h, dA, m, n, ld, n, dP, dQ);
        if (rc) return rc;
        CK(cudaMemcpyAsync(A, dA, (size_t)m * ld * 8, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(Q, dQ, (size_t)qn * 8, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(rank, r_dev(h), 8, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaMemcpyAsync(P, dP, (size_t)m * 8, cudaMemcpyDeviceToHost, h->stream));
    return finish_sync(h);
}

int gf2_rref_host(gf2_handle_t h, uint64_t *A, int64_t m, int64_t n, int64_t ld, int64_t *Q, int64_t *rank)
{
    int rc = check_args(h, A, m, n, ld);
    if (rc) return rc;
    if (!rank || (m > 0 && n > 0 && !Q)) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    *rank = 0;
    if (m == 0 || n == 0) return GF2_OK;
    const int64_t qn = std::min(m, n);
    const size_t abytes = align256((size_t)m * ld * 8);
    const size_t need = abytes + align256((size_t)qn * 8);
    rc = grow(&h->io, &h->io_cap, need, h->stream);
    if (rc) return rc;
    uint64_t *dA = reinterpret_cast<uint64_t *>(h->io);
    int64_t *dQ = reinterpret_cast<int64_t *>(h->io + abytes);
    CK(cudaMemcpyAsync(dA, A, (size_t)m * ld * 8, cudaMemcpyHostToDevice, h->stream));
    rc = rref_enqueue(h, dA, m, n, ld, dQ);
    if (rc) return rc;
    CK(cudaMemcpyAsync(A, dA, (size_t)m * ld * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(Q, dQ, (size_t)qn * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(rank, r_dev(h), 8, cudaMemcpyDeviceToHost, h->stream));
    return finish_sync(h);
}

int gf2_selftest_wait(gf2_handle_t h, int64_t limit_us)
{
    if (!h || limit_us < 0 || limit_us > 1000000) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    CK(launch_wait_selftest(h->stream, err_dev(h), (unsigned long long)limit_us * 1000ull));
    h->launches += 1;
    return finish_sync(h);
}

int gf2_set_option(gf2_handle_t h, int option, int64_t value)
{
    if (!h) return GF2_EINVAL;
    switch (option) {
    case GF2_OPT_LOOKAHEAD: h->lookahead = value != 0; return GF2_OK;
    case GF2_OPT_TC_MUL: h->tc_mul = value != 0; return GF2_OK;
    case GF2_OPT_TC_UPDATE: h->tc_update = value != 0; return GF2_OK;
    case GF2_OPT_TMA_UPDATE: h->tma = value != 0; return GF2_OK;
    case GF2_OPT_PLE_BLOCK:
        if (value < -1 || (value > 0 && value % 64)) return GF2_EINVAL;
        h->ple_block = value;
        return GF2_OK;
    case GF2_OPT_RREF_BLOCK:
        if (value < -1 || (value > 0 && value % 64)) return GF2_EINVAL;
        h->rref_block = value;
        return GF2_OK;
    case GF2_OPT_WIDE_UPDATE: h->wide_update = value != 0; return GF2_OK;
    case GF2_OPT_NAIVE_UPDATE: h->naive_update = value != 0; return GF2_OK;
    case GF2_OPT_PDL: h->pdl = value != 0; return GF2_OK;
    case GF2_OPT_PLE_RECURSIVE: h->ple_recursive = value != 0; return GF2_OK;
    case GF2_OPT_RREF_LEAF: h->rref_leaf = value != 0; return GF2_OK;
    case GF2_OPT_RREF_COMPACT: h->rref_compact = value != 0; return GF2_OK;
    case GF2_OPT_TRSM_LEAF:
        if (value != 1024 && value != 2048 && value != 4096) return GF2_EINVAL;
        h->leaf_rows = value;
        return GF2_OK;
    case GF2_OPT_MUL_GEMM_FORMAT:
        if (value != 8 && value != 4 && value != 0) return GF2_EINVAL;
        if (value != 0 && !kLibraryGemm) return GF2_EINVAL;   // library GEMM not built in
        h->gemm_fmt = (int)value;
        return GF2_OK;
    case GF2_OPT_MUL_GEMM_MIN_K:
        if (value < 0) return GF2_EINVAL;
        h->gemm_min_k = value;
        return GF2_OK;
    default: return GF2_EINVAL;
    }
}

int gf2_set_profiling(gf2_handle_t h, int on)
{
    if (!h) return GF2_EINVAL;
    h->profiling = on < 0 ? 0 : (on > 5 ? 5 : on);
    return GF2_OK;
}

int gf2_get_stats(gf2_handle_t h, gf2_stats *out)
{
    if (!h || !out) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    CK(cudaStreamSynchronize(h->stream));
    for (auto &p : h->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) h->kind_ms[p.kind] += ms;
        else cudaGetLastError();
        if (h->profiling == 4) {
            float t0 = 0.f, t1 = 0.f;
            if (!h->tl_ref) h->tl_ref = p.e0;           // kept as the origin until the next reset
            if (cudaEventElapsedTime(&t0, h->tl_ref, p.e0) == cudaSuccess &&
                cudaEventElapsedTime(&t1, h->tl_ref, p.e1) == cudaSuccess) {
                h->timeline.push_back((double)p.kind);
                h->timeline.push_back((double)t0);
                h->timeline.push_back((double)t1);
            } else {
                cudaGetLastError();
            }
        }
        if (p.e0 != h->tl_ref) h->ev_free.push_back(p.e0);
        h->ev_free.push_back(p.e1);
    }
    h->ev_pending.clear();
    unsigned long long bytes = 0;
    int32_t fb = 0;
    CK(cudaMemcpy(&bytes, bytes_dev(h), 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&fb, fb_dev(h), 4, cudaMemcpyDeviceToHost));
    out->kernel_launches = h->launches;
    out->update_launches = h->upd_launches;
    out->update_timed_launches = h->upd_timed;
    out->update_ms = h->kind_ms[K_UPDATE];
    out->panel_ms = h->kind_ms[K_PANEL];
    out->prep_ms = h->kind_ms[K_PREP];
    out->rref_prep_ms = h->kind_ms[K_RPREP];
    out->other_ms = h->kind_ms[K_OTHER];
    out->rref_pass_ms = h->kind_ms[K_RPASS];
    out->rref_pass_launches = h->rpass_launches;
    out->rref_pass_timed_launches = h->rpass_timed;
    unsigned long long b2 = 0;
    CK(cudaMemcpy(&b2, h->small + SM_BYTES2, 8, cudaMemcpyDeviceToHost));
    out->rref_pass_bytes = (double)b2;
    out->gemm_ms = h->kind_ms[K_GEMM];
    out->gemm_flops = h->gemm_flops;
    out->gemm_launches = h->gemm_launches;
    out->gemm_timed_launches = h->gemm_timed;
    out->gemm_flops_all = h->gemm_flops_all;
    out->update_bytes = (double)bytes;
    out->panel_fallbacks = fb;
    return GF2_OK;
}

int gf2_get_timeline(gf2_handle_t h, double *out, int64_t max_records, int64_t *count)
{
    if (!h || !count || max_records < 0 || (max_records > 0 && !out)) return GF2_EINVAL;
    gf2_stats st;
    const int rc = gf2_get_stats(h, &st);                 // resolves the pending events
    if (rc) return rc;
    const int64_t n = (int64_t)h->timeline.size() / 3;
    *count = n;
    const int64_t k = std::min(n, max_records);
    for (int64_t i = 0; i < 3 * k; ++i) out[i] = h->timeline[(size_t)i];
    return GF2_OK;
}

int gf2_reset_stats(gf2_handle_t h)
{
    if (!h) return GF2_EINVAL;
    DeviceGuard g(h->device);
    PdlScope pdl_scope(h->pdl);
    CK(cudaStreamSynchronize(h->stream));
    for (auto &p : h->ev_pending) { h->ev_free.push_back(p.e0); h->ev_free.push_back(p.e1); }
    h->ev_pending.clear();
    if (h->tl_ref) { h->ev_free.push_back(h->tl_ref); h->tl_ref = nullptr; }
    h->timeline.clear();
    h->launches = 0;
    h->upd_launches = 0;
    h->upd_timed = 0;
    h->rpass_launches = 0;
    h->rpass_timed = 0;
    h->gemm_launches = 0;
    h->gemm_timed = 0;
    h->gemm_flops = 0.0;
    h->gemm_flops_all = 0.0;
    CK(cudaMemset(h->small + SM_BYTES2, 0, 8));
    for (double &x : h->kind_ms) x = 0.0;
    CK(cudaMemset(h->small + SM_FALLBACK, 0, 12));
    return GF2_OK;
}

const char *gf2_strerror(int code)
{
    switch (code) {
    case GF2_OK: return "GF2_OK";
    case GF2_EINVAL: return "GF2_EINVAL: invalid argument";
    case GF2_ENOMEM: return "GF2_ENOMEM: device allocation failed";
    case GF2_ECUDA: return "GF2_ECUDA: CUDA runtime error";
    case GF2_ETIMEOUT: return "GF2_ETIMEOUT: bounded device wait ran out";
    case GF2_EINTERNAL: return "GF2_EINTERNAL: device-side consistency check failed";
    default: return "GF2: unknown status";
    }
}

}  // extern "C"
