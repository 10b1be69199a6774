// noalloc.cu -- gf2_ple_noalloc: the PLE decomposition without any device
// memory allocation.
//
// Who needs this: callers that cannot call cudaMalloc.  A serving process or
// a framework that hands all of the GPU's memory to its own allocator at
// start-up has nothing left for a library to allocate, and code that must not
// stall cannot afford cudaMalloc / cudaFree, which may wait for other work on
// the device.  Such callers pass their own input and output buffers and get
// the same result as gf2_ple, with every piece of scratch memory the kernels
// need taken from one fixed array that is part of the library image.
//
// The scratch is the file-scope __device__ array below.  Every GPU that loads
// the library holds it (NA_BYTES, about 0.5 MiB) until the process exits.  In
// host code the array's name is only a host-side stand-in, so the address the
// kernels get comes from cudaGetSymbolAddress, looked up once per device (on
// the first call made with that device current) and cached.
//
// All calls share the one array, which keeps whatever the last call left in
// it; each call re-initialises everything that must start in a known state
// (running rank, row map, error flag).  Two calls whose work overlaps on the
// GPU -- on different streams, or on different host threads without ordering
// -- race on the array and may return wrong results.
#include "common.cuh"
#include "gf2.h"

#include <mutex>

namespace {

using namespace gf2;

constexpr int64_t NA_MAX_ROWS = 4096;
constexpr int64_t NA_MAX_COLS = 4096;
constexpr int64_t NA_W = NA_MAX_COLS / 64;
constexpr int64_t NA_LDS = NA_W + (NA_W & 1);

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_SMALL = 0;  // int64 rank, int32 error flag, int32 fallback counter
constexpr size_t OFF_DESC = al256(OFF_SMALL + 64);
constexpr size_t OFF_IDX = al256(OFF_DESC + (size_t)NA_W * sizeof(StripeDesc));
constexpr size_t OFF_MAP = al256(OFF_IDX + (size_t)NA_MAX_ROWS * 8);
constexpr size_t OFF_S = al256(OFF_MAP + (size_t)NA_MAX_ROWS * 4);
constexpr size_t OFF_GVAL = al256(OFF_S + (size_t)SMAX * NA_LDS * 8);
constexpr size_t OFF_GLB = al256(OFF_GVAL + (size_t)NA_MAX_ROWS * 8);
constexpr size_t OFF_GSRC = al256(OFF_GLB + (size_t)NA_MAX_ROWS * 8);
constexpr size_t OFF_GPOS = al256(OFF_GSRC + (size_t)NA_MAX_ROWS * 4);
constexpr size_t OFF_PTAB = al256(OFF_GPOS + (size_t)NA_MAX_ROWS * 4);
constexpr size_t NA_BYTES = al256(OFF_PTAB + PREP_TAB_BYTES);

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

struct NoallocDevice {
    bool ready = false;
    char *base = nullptr;   // device address of g_noalloc_scratch on this device
    int num_sms = 1;
};
constexpr int NA_MAX_DEVICES = 64;
NoallocDevice g_na_dev[NA_MAX_DEVICES];
std::mutex g_na_mu;

// Once per device, with that device current: resolve the array's device
// address and prepare the update kernel's shared-memory limit.
int noalloc_setup(int dev, NoallocDevice **out)
{
    std::lock_guard<std::mutex> lk(g_na_mu);
    NoallocDevice &d = g_na_dev[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return GF2_ECUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return GF2_ECUDA;
        }
        if (setup_update_kernel() != cudaSuccess) {
            cudaGetLastError();
            return GF2_ECUDA;
        }
        d.base = static_cast<char *>(ptr);
        d.num_sms = sms;
        d.ready = true;
    }
    *out = &d;
    return GF2_OK;
}

#define NA_CK(expr)                                                      \
    do {                                                                 \
        if ((expr) != cudaSuccess) { cudaGetLastError(); return GF2_ECUDA; } \
    } while (0)

}  // namespace

extern "C" int gf2_ple_noalloc(uint64_t *A, int64_t m, int64_t n, int64_t ld_words, int64_t *P,
                               int64_t *Q, int64_t *rank, void *stream)
{
    if (!rank || m < 0 || n < 0) return GF2_EINVAL;
    if (m > NA_MAX_ROWS || n > NA_MAX_COLS) return GF2_EINVAL;   // beyond the fixed scratch
    const int64_t W = (n + 63) / 64;
    if (m > 0 && n > 0 && (!A || !P || !Q || ld_words < W)) return GF2_EINVAL;
    if (m > 0 && !P) return GF2_EINVAL;
    *rank = 0;
    if (m == 0) return GF2_OK;

    // the call synchronises the stream between launches: it cannot be
    // captured (checked first: no other runtime call happens on a stream that
    // is capturing)
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NA_CK(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return GF2_EINVAL;
    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return GF2_EINVAL;
    NoallocDevice *nd = nullptr;
    int rc = noalloc_setup(dev, &nd);
    if (rc) return rc;
    // the scratch address is the current device's: the work must run there
    int sdev = dev;
    NA_CK(cudaStreamGetDevice(st, &sdev));
    if (sdev != dev) return GF2_EINVAL;

    char *base = nd->base;
    int64_t *r_dev = reinterpret_cast<int64_t *>(base + OFF_SMALL);
    int32_t *err = reinterpret_cast<int32_t *>(base + OFF_SMALL + 8);
    int32_t *fallbacks = reinterpret_cast<int32_t *>(base + OFF_SMALL + 12);
    StripeDesc *descs = reinterpret_cast<StripeDesc *>(base + OFF_DESC);
    uint64_t *IDX = reinterpret_cast<uint64_t *>(base + OFF_IDX);
    int32_t *map = reinterpret_cast<int32_t *>(base + OFF_MAP);
    uint64_t *S = reinterpret_cast<uint64_t *>(base + OFF_S);
    PanelScratch gs{reinterpret_cast<uint64_t *>(base + OFF_GVAL), reinterpret_cast<uint64_t *>(base + OFF_GLB),
                    reinterpret_cast<int32_t *>(base + OFF_GSRC), reinterpret_cast<int32_t *>(base + OFF_GPOS)};

    // what must start from a known state: error flag and counters (the rank
    // and the row map are reset by the init kernel)
    NA_CK(cudaMemsetAsync(base + OFF_SMALL, 0, 64, st));
    NA_CK(launch_init_ple(st, P, Q, m, n > 0 ? (m < n ? m : n) : 0, map, r_dev, nd->num_sms));
    const int64_t ns = W;
    for (int64_t s = 0; s < ns; ++s) {
        uint64_t *ptab = reinterpret_cast<uint64_t *>(base + OFF_PTAB);
        NA_CK(launch_panel(st, A, m, ld_words, n, (int)s, descs, r_dev, P, Q, map, gs, fallbacks, ptab));
        NA_CK(launch_prep(st, A, m, ld_words, W, (int)s, descs, map, S, NA_LDS, IDX, err, ptab, nd->num_sms));
        UpdArgs a{};
        a.tp_lo = 0;
        a.tp_hi = -1;
        a.left_copies = 1;
        a.mode = UPD_PLE;
        a.A = A;
        a.ld = ld_words;
        a.m = m;
        a.W = W;
        a.desc = descs + s;
        a.stripe = (int)s;
        a.S = S;
        a.ldS = NA_LDS;
        a.map = map;
        a.idx = IDX;
        a.idx_stride = 1;
        a.bytes = nullptr;
        NA_CK(launch_update(st, a, nd->num_sms));
    }
    int64_t r = 0;
    int32_t e = 0;
    NA_CK(cudaMemcpyAsync(&r, r_dev, sizeof(r), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaMemcpyAsync(&e, err, sizeof(e), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (e) return GF2_EINTERNAL;
    *rank = r;
    return GF2_OK;
}
