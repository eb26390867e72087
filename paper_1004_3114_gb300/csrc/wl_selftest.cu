// Self-test of the bounded device-side wait that every mbarrier wait of the
// bulk-copy kernels goes through (mbar_wait, wl_tma_common.cuh): one CTA
// waits on a barrier that nothing ever arrives at and must give up after the
// cycle budget (about a second) instead of hanging, then waits on a barrier
// whose phase has completed and must return at once.  No memory is touched
// out of bounds and nothing is left waiting, so the context stays usable.
#include <cuda_runtime.h>

#include "wallace.h"
#include "wl_tma_common.cuh"

namespace {

__global__ void bounded_wait_kernel(int *result)
{
    using namespace wl_tma;
    __shared__ __align__(8) uint64_t bar_never, bar_done;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar_never), 1);
        mbar_init(smem_u32(&bar_done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        mbar_arrive(smem_u32(&bar_done));   // phase 0 of this one completes
        const bool never = mbar_wait(smem_u32(&bar_never), 0u);
        const bool done = mbar_wait(smem_u32(&bar_done), 0u);
        result[0] = never ? 0 : WALLACE_ETIMEOUT;
        result[1] = done ? 1 : 0;
    }
}

} // namespace

extern "C" int wallace_selftest_bounded_wait(int *completed_ok)
{
    int *d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess)
        return WALLACE_ECUDA;
    int h[2] = {0, 0};
    cudaError_t e = cudaMemset(d, 0, 2 * sizeof(int));
    if (e == cudaSuccess) {
        bounded_wait_kernel<<<1, 32>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess)
        return WALLACE_ECUDA;
    if (completed_ok)
        *completed_ok = h[1];
    return h[0];
}
