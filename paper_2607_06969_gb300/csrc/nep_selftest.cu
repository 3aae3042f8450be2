// Self-test of the bounded tensor-core completion wait used by the
// mixed-precision angular kernel: the timeout path in isolation.
#include "nep_internal.h"
#include "nep_tmem.cuh"

namespace nep {
namespace {

// one CTA: tensor memory allocated, an mbarrier expecting one arrival that
// never comes, a bounded wait, the outcome in *flag (1 completed, 2 timed
// out), the columns freed
__global__ void __launch_bounds__(128) k_wait_selftest(int polls, int* flag) {
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tc5::alloc(&slot, 32);
    if (threadIdx.x == 0) tc5::mbar_init(&bar, 1);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const bool got = tc5::mbar_wait(&bar, 0, polls);
    const bool all = __syncthreads_and(got);
    if (threadIdx.x == 0) atomicOr(flag, all ? 1 : 2);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (warp == 0) tc5::dealloc(slot, 32);
}

}  // namespace

cudaError_t wait_selftest(cudaStream_t st, int* outcome) {
    int* flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e) return e;
    if (!(e = cudaMemsetAsync(flag, 0, sizeof(int), st))) {
        k_wait_selftest<<<1, 128, 0, st>>>(1000, flag);
        if (!(e = cudaGetLastError()) && !(e = cudaStreamSynchronize(st)))
            e = cudaMemcpy(outcome, flag, sizeof(int), cudaMemcpyDeviceToHost);
    }
    cudaFree(flag);
    return e;
}

}  // namespace nep
