// server.cu -- a continuous-batching request loop for GF(2) solve jobs.
//
// Section 1 names solving dense systems as the use of the decomposition; this
// is the serving side of that: jobs arrive over time, each a system A X = B
// in host memory.  The server owns `slots` execution slots (a CUDA stream, a
// gf2 handle and device buffers sized once at start-up for the largest job),
// each driven by its own thread.  Whenever a slot is free and the job at the
// head of the queue fits in the remaining HBM budget, the slot takes it: its
// inputs are copied in, gf2_solve_async runs on the slot's stream, and the
// solution and status are copied back.  Jobs admitted while others are
// running therefore overlap on the device; results are handed to the caller
// through gf2_server_poll.  Nothing in the loop allocates device memory after
// start-up.
#include "gf2.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

inline int64_t words_of(int64_t n) { return (n + 63) >> 6; }

struct Slot {
    gf2_handle_t h = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    uint64_t *dA = nullptr, *dB = nullptr;
    int32_t *dstatus = nullptr;
    int32_t *hstatus = nullptr;       // pinned
    size_t footprint = 0;
};

struct Pending {
    gf2_solve_job job;
    double t_submit;
};

}  // namespace

struct gf2_server {
    int device = 0;
    int64_t max_n = 0, max_nrhs = 0;
    size_t budget = 0, in_use = 0;
    std::vector<Slot> slots;
    std::deque<Pending> queue;
    std::vector<gf2_solve_result> finished;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    std::atomic<bool> stop{false};
    int64_t submitted = 0, completed = 0;
};

namespace {

size_t job_footprint(const gf2_solve_job &j)
{
    // device bytes the job occupies while it runs: A, B and the solve's
    // augmented copy and workspace (about twice A)
    const size_t a = (size_t)j.n * words_of(j.n) * 8;
    const size_t b = (size_t)j.n * std::max<int64_t>(words_of(j.nrhs), 1) * 8;
    return 3 * a + 2 * b;
}

// Run one job on a slot, synchronously on the slot's stream (slot thread).
int run_job(Slot &sl, const gf2_solve_job &j)
{
    const int64_t wa = words_of(j.n), wb = std::max<int64_t>(words_of(j.nrhs), 1);
    int rc = GF2_OK;
    if (cudaMemcpy2DAsync(sl.dA, wa * 8, j.A, j.lda * 8, wa * 8, j.n, cudaMemcpyHostToDevice, sl.st) != cudaSuccess ||
        (j.nrhs > 0 && cudaMemcpy2DAsync(sl.dB, wb * 8, j.B, j.ldb * 8, words_of(j.nrhs) * 8, j.n,
                                         cudaMemcpyHostToDevice, sl.st) != cudaSuccess))
        rc = GF2_ECUDA;
    if (!rc) rc = gf2_solve_async(sl.h, sl.dA, j.n, wa, sl.dB, j.nrhs, wb, sl.dstatus);
    if (!rc && j.nrhs > 0 && j.X &&
        cudaMemcpy2DAsync(j.X, j.ldx * 8, sl.dB, wb * 8, words_of(j.nrhs) * 8, j.n, cudaMemcpyDeviceToHost,
                          sl.st) != cudaSuccess)
        rc = GF2_ECUDA;
    if (!rc && cudaMemcpyAsync(sl.hstatus, sl.dstatus, 4, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
        rc = GF2_ECUDA;
    if (!rc && cudaStreamSynchronize(sl.st) != cudaSuccess) rc = GF2_ECUDA;
    if (rc) cudaGetLastError();
    return rc;
}

// One thread per slot: take the head of the queue whenever this slot is free
// and the job fits in the HBM budget (a job always runs if nothing else
// does), run it, publish the result.  Each slot issuing its own launches
// keeps the host from serialising the jobs' kernel launches.
void slot_loop(gf2_server *s, int idx)
{
    cudaSetDevice(s->device);
    Slot &sl = s->slots[idx];
    while (true) {
        Pending p;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] {
                if (s->queue.empty()) return s->stop.load();
                const size_t fp = job_footprint(s->queue.front().job);
                return s->in_use == 0 || s->in_use + fp <= s->budget;
            });
            if (s->queue.empty()) return;              // stopping and nothing left
            p = s->queue.front();
            s->queue.pop_front();
            sl.footprint = job_footprint(p.job);
            s->in_use += sl.footprint;
        }
        const double t_start = now_s();
        const int rc = run_job(sl, p.job);
        gf2_solve_result res{};
        res.id = p.job.id;
        res.status = rc ? -1 : *sl.hstatus;
        res.error = rc;
        res.t_submit = p.t_submit;
        res.t_start = t_start;
        res.t_done = now_s();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->finished.push_back(res);
            s->in_use -= sl.footprint;
            s->completed += 1;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();                       // the budget freed up
    }
}

void destroy_slots(gf2_server *s)
{
    for (Slot &sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.h) gf2_destroy(sl.h);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
        cudaFree(sl.dA);
        cudaFree(sl.dB);
        cudaFree(sl.dstatus);
        if (sl.hstatus) cudaFreeHost(sl.hstatus);
    }
    s->slots.clear();
}

}  // namespace

extern "C" {

int gf2_server_create(gf2_server_t *out, int device, int slots, int64_t max_n, int64_t max_nrhs,
                      size_t hbm_budget_bytes)
{
    if (!out || slots < 1 || slots > 64 || max_n < 1 || max_nrhs < 0) return GF2_EINVAL;
    *out = nullptr;
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return GF2_ECUDA;
    if (cudaSetDevice(dev) != cudaSuccess) { cudaGetLastError(); return GF2_ECUDA; }
    gf2_server *s = new (std::nothrow) gf2_server();
    if (!s) return GF2_ENOMEM;
    s->device = dev;
    s->max_n = max_n;
    s->max_nrhs = max_nrhs;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)-1;
    s->slots.resize(slots);
    const int64_t wa = words_of(max_n), wb = std::max<int64_t>(words_of(max_nrhs), 1);
    int rc = GF2_OK;
    for (Slot &sl : s->slots) {
        if (gf2_create(&sl.h, dev) != GF2_OK || cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&sl.dA, (size_t)max_n * wa * 8) != cudaSuccess ||
            cudaMalloc(&sl.dB, (size_t)max_n * wb * 8) != cudaSuccess ||
            cudaMalloc(&sl.dstatus, 4) != cudaSuccess || cudaMallocHost(&sl.hstatus, 4) != cudaSuccess) {
            cudaGetLastError();
            rc = GF2_ENOMEM;
            break;
        }
        gf2_set_stream(sl.h, sl.st);
        // size the handle's workspace for the largest job now, not in the loop
        cudaMemsetAsync(sl.dA, 0, (size_t)max_n * wa * 8, sl.st);
        cudaMemsetAsync(sl.dB, 0, (size_t)max_n * wb * 8, sl.st);
        rc = gf2_solve_async(sl.h, sl.dA, max_n, wa, sl.dB, max_nrhs, wb, sl.dstatus);
        if (rc || cudaStreamSynchronize(sl.st) != cudaSuccess) { cudaGetLastError(); rc = rc ? rc : GF2_ECUDA; break; }
    }
    if (rc) {
        destroy_slots(s);
        delete s;
        return rc;
    }
    for (int i = 0; i < slots; ++i) s->workers.emplace_back(slot_loop, s, i);
    *out = s;
    return GF2_OK;
}

int gf2_server_submit(gf2_server_t s, const gf2_solve_job *job)
{
    if (!s || !job || job->n < 0 || job->n > s->max_n || job->nrhs < 0 || job->nrhs > s->max_nrhs) return GF2_EINVAL;
    if (job->n > 0 && (!job->A || job->lda < words_of(job->n))) return GF2_EINVAL;
    if (job->n > 0 && job->nrhs > 0 && (!job->B || job->ldb < words_of(job->nrhs))) return GF2_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.push_back({*job, now_s()});
        s->submitted += 1;
    }
    s->cv_work.notify_one();
    return GF2_OK;
}

int gf2_server_poll(gf2_server_t s, gf2_solve_result *out, int max_results, int *count)
{
    if (!s || !count || max_results < 0 || (max_results > 0 && !out)) return GF2_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const int k = (int)std::min<size_t>((size_t)max_results, s->finished.size());
    for (int i = 0; i < k; ++i) out[i] = s->finished[i];
    s->finished.erase(s->finished.begin(), s->finished.begin() + k);
    *count = k;
    return GF2_OK;
}

int gf2_server_drain(gf2_server_t s)
{
    if (!s) return GF2_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->completed == s->submitted; });
    return GF2_OK;
}

double gf2_server_clock(void) { return now_s(); }

int gf2_server_destroy(gf2_server_t s)
{
    if (!s) return GF2_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop.store(true);
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers)
        if (t.joinable()) t.join();
    cudaSetDevice(s->device);
    destroy_slots(s);
    delete s;
    return GF2_OK;
}

}  // extern "C"
