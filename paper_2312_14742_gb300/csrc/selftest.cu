// Self-test of the failure detection of the staged kernels: a wait on an
// mbarrier whose phase nothing completes, with the same bounded wait and the
// same device counter as the step kernels, so that a test or a health check
// can see a wait run out and reach the host as LBM_ETIMEOUT without any fault.
#include "kernels.h"
#include "tma.cuh"

namespace lbm {

namespace {

__global__ void wait_timeout_kernel(unsigned int* timeouts)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival expected; none comes
        mbar_init_fence();
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0) && threadIdx.x == 0) atomicAdd(timeouts, 1u);
}

}  // namespace

cudaError_t launch_selftest_timeout(unsigned int* timeouts, cudaStream_t s)
{
    if (!timeouts) return cudaErrorInvalidValue;
    wait_timeout_kernel<<<1, 32, 0, s>>>(timeouts);
    return cudaGetLastError();
}

}  // namespace lbm
