// selftest.cu -- exercises the bounded device-side wait that the tcgen05 and
// TMA kernels use, without any fault: one CTA initialises an mbarrier that
// nothing will ever arrive on, waits for it with the same bounded wait, and
// records the expiry in the handle's error word, exactly as those kernels do
// when a copy or a product never completes.  The host then reports
// GF2_ETIMEOUT and the context stays usable.
#include "async_dev.cuh"
#include "common.cuh"

namespace gf2 {

__global__ void wait_selftest_kernel(int32_t *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init_cta(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    // no thread arrives: the wait can only end by its limit
    if (!mbar_wait_limited(&bar, 0u, limit_ns) && threadIdx.x == 0) atomicExch(err, 4);   // GF2_ETIMEOUT
}

cudaError_t launch_wait_selftest(cudaStream_t st, int32_t *err, unsigned long long limit_ns)
{
    wait_selftest_kernel<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

}  // namespace gf2
