// Grid-wide synchronisation for kernels that run many passes of one pool in a
// single cooperative launch (every CTA resident): a bounded grid barrier per
// pass, the pass's exact sum of squares gathered from every CTA into one of
// three rotating accumulator sets, and (for kernels that deal tiles
// dynamically) three rotating tile counters.  Set p mod 3 serves pass p; a
// set is zeroed during the pass before it is used, by which time every CTA
// has passed the barrier that ended its previous use, so no zeroing races a
// reader.  The device scratch is zeroed by the host before each launch.
#pragma once

#include <stdint.h>

#include "wl_common.cuh"

#define WL_GRID_WAIT_CYCLES 2000000000ll   /* about one second */

namespace {

struct WlGridAcc {
    alignas(128) unsigned long long a0, a1, a2;   // Q limbs: bits 0-31, 32-63, 64-127 of CTA sums
    unsigned int bad;
};

struct alignas(128) WlGridCtr {
    unsigned int v;
};

struct WlGridSync {
    alignas(128) unsigned int arrived;   // barrier arrivals so far
    alignas(128) int abort;              // a CTA gave up waiting
    WlGridAcc acc[3];                    // sum of squares of pass p in set p mod 3
    WlGridCtr ctr[3];                    // tiles dealt in pass p, counter p mod 3
};

__device__ __forceinline__ unsigned int wl_ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Arrival at the grid barrier (thread 0, after a CTA barrier that follows
// the CTA's writes of the pass): its release publishes them.
__device__ __forceinline__ void wl_grid_arrive(WlGridSync *sy)
{
    if (threadIdx.x == 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(&sy->arrived) : "memory");
}

// Bounded wait for `target` arrivals: true when every CTA has arrived, false
// when the wait gave up or another CTA did.  Every thread calls.
__device__ bool wl_grid_wait(WlGridSync *sy, unsigned int target)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        int ok = 1;
        while (wl_ld_acquire_u32(&sy->arrived) < target) {
            if (*(volatile int *)&sy->abort || clock64() - t0 > WL_GRID_WAIT_CYCLES) {
                ok = 0;
                atomicExch(&sy->abort, 1);
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// CTA sum of (lo, hi, bad) into one accumulator set (every thread calls;
// `red` holds 3 words per warp).
__device__ void wl_grid_reduce_to(uint64_t lo, uint64_t hi, uint32_t bad, WlGridAcc *acc, uint64_t *red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const uint64_t olo = __shfl_down_sync(0xffffffffu, lo, off);
        const uint64_t ohi = __shfl_down_sync(0xffffffffu, hi, off);
        wl_add128(lo, hi, olo, ohi);
    }
    bad = __any_sync(0xffffffffu, bad) ? 1u : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        red[warp] = lo;
        red[nw + warp] = hi;
        red[2 * nw + warp] = bad;
    }
    __syncthreads();
    if (warp == 0) {
        lo = lane < nw ? red[lane] : 0ull;
        hi = lane < nw ? red[nw + lane] : 0ull;
        bad = lane < nw ? (uint32_t)red[2 * nw + lane] : 0u;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const uint64_t olo = __shfl_down_sync(0xffffffffu, lo, off);
            const uint64_t ohi = __shfl_down_sync(0xffffffffu, hi, off);
            wl_add128(lo, hi, olo, ohi);
        }
        bad = __any_sync(0xffffffffu, bad) ? 1u : 0u;
        if (lane == 0) {
            atomicAdd(&acc->a0, (unsigned long long)(lo & 0xffffffffull));
            atomicAdd(&acc->a1, (unsigned long long)(lo >> 32));
            if (hi)
                atomicAdd(&acc->a2, (unsigned long long)hi);
            if (bad)
                atomicOr(&acc->bad, 1u);
        }
    }
    __syncthreads();
}

// Q of a set as a 128-bit integer (lo, hi) and its bad flag, read by one
// thread after the grid barrier of the set's pass.
__device__ __forceinline__ void wl_grid_q(const WlGridAcc *acc, uint64_t &lo, uint64_t &hi, uint32_t &bad)
{
    const unsigned long long a0 = __ldcg(&acc->a0), a1 = __ldcg(&acc->a1), a2 = __ldcg(&acc->a2);
    bad = __ldcg(&acc->bad);
    const unsigned long long t = a0 + (a1 << 32);
    hi = a2 + (a1 >> 32) + (t < a0 ? 1ull : 0ull);
    lo = t;
}

} // namespace
