// Failure-path self-test of the bounded waits: one block initialises an
// mbarrier that nothing ever arrives at and waits on it with the sweeps' wait
// helper; the wait gives up after its poll bound, the block raises
// FLAG_TIMEOUT and returns, and the next synchronising call reports
// PPMLR_E_TIMEOUT with the context still usable.
#include "sweep.cuh"

namespace ppmlr {

__global__ void __launch_bounds__(32) wait_selftest_kernel(int *flags, int polls)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool done = mbar_wait(&bar, 0u, polls);     // no arrival: the phase never completes
    if (!done && threadIdx.x == 0) atomicOr(flags, FLAG_TIMEOUT);
}

cudaError_t launch_wait_selftest(int *flags, int polls, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(flags, polls);
    return cudaGetLastError();
}

}  // namespace ppmlr
