// Pieces of the warp-specialised bulk-copy (TMA) pass shared by the
// grid-wide pass kernel (wl_tiled_tma.cu) and the CTA-local runner of the
// batched generators (wl_tma_run.cuh): launch shape, stage ring layout,
// mbarrier and bulk-copy wrappers, the exact sum-of-squares term, and
// divisions by the lane and span counts of the lane-tiled geometry.
#pragma once

#include <stdint.h>

#include "wl_common.cuh"

#define TM_CONS_WARPS 15          /* 45 lanes = 3 per consumer warp */
#define TM_CONS_THREADS (TM_CONS_WARPS * 32)
#define TM_PROD_WARPS 4          /* one warp issues a bulk copy only every ~80 cycles */
#define TM_THREADS (TM_CONS_THREADS + 32 * TM_PROD_WARPS)
#define TM_STAGES 3               /* n = 4: ring stages */
#define TM_ETARGET 2880          /* n = 4: lane-times per tile, L * T <= this (T = 64 at L = 45) */
#define TM_STAGES2 2              /* n = 2: ring stages */
#define TM_ETARGET2 11520        /* n = 2: lane-times per tile (T = 192 to 512 at L = 55 to 21) */
#define TM_LMAX 45               /* n = 4: strides divide 45 */
#define TM_LMAX2 55              /* n = 2: L = alpha beta <= 5 * 11 */
#define TM_MAXSPANS 32           /* sum_i 45 / alpha_i <= 15 + 9 + 5 + 3 */
#define TM_MIN_N 16384
#define TM_WAIT_CYCLES 2000000000ll   /* about one second */

namespace wl_tma {


// Ring geometry of the pass kernel per sub-vector count: n = 4 keeps three
// stages of 2880 lane-times (45 lanes x 64); n = 2 has two stages of twice
// the values (lanes of 192 to 512 times fill its 64-time items better).
template <int NSUB>
__host__ __device__ constexpr int tm_stages() { return NSUB == 4 ? TM_STAGES : TM_STAGES2; }
template <int NSUB>
__host__ __device__ constexpr int tm_et() { return NSUB == 4 ? TM_ETARGET : TM_ETARGET2; }
template <int NSUB>
__host__ __device__ constexpr int tm_stage_data_words() { return NSUB * tm_et<NSUB>() + 12 * TM_MAXSPANS; }
template <int NSUB>
__host__ __device__ constexpr int tm_stage_words() { return tm_stage_data_words<NSUB>() + TM_MAXSPANS; }
// common area: J[L + 1] (room for n = 2's 55 lanes), lane table (n * lanes <= 180), span starts
__host__ __device__ constexpr int tm_common_words() { return (TM_LMAX2 + 1) + 4 * TM_LMAX + TM_MAXSPANS; }
template <int NSUB>
__host__ __device__ constexpr size_t tm_smem_bytes()
{
    return sizeof(float) * (size_t)(tm_stages<NSUB>() * tm_stage_words<NSUB>() + tm_common_words());
}

// x / d for x >= 0 and d a lane count or span count of either geometry
// (divisors of 45; 3, 5, 7, 11 and their products for n = 2): constant
// divisors, so each case is a multiply and shift instead of a division
// routine
__device__ __forceinline__ int tm_divc(int x, int d)
{
    switch (d) {
    case 7:
        return x / 7;
    case 11:
        return x / 11;
    case 21:
        return x / 21;
    case 33:
        return x / 33;
    case 35:
        return x / 35;
    case 55:
        return x / 55;
    case 1:
        return x;
    case 3:
        return x / 3;
    case 5:
        return x / 5;
    case 9:
        return x / 9;
    case 15:
        return x / 15;
    case 45:
        return x / 45;
    default:
        return x / d;
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(bar)
                 : "memory");
}

// true when the phase with the given parity has completed; false after the
// cycle budget runs out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long start = clock64();
    while (true) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done)
            return true;
        if (clock64() - start > TM_WAIT_CYCLES)
            return false;
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// floor(y^2 2^32) of one binary32 value, exact.  y = m 2^(e-150) with the
// hidden bit in m, so y^2 2^32 = m^2 / 2^(268-2e).  The shift is clamped to
// 63 as an unsigned value: e <= 110 (|y| < 2^-16) gives 0, and e >= 135
// (|y| >= 256, Inf, NaN: a corrupt pool) wraps to a huge shift and also
// gives 0; such exponents are caught through the running maximum `emax`.
__device__ __forceinline__ uint64_t term32(float y, uint32_t &emax)
{
    const uint32_t u = __float_as_uint(y);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint32_t m = (u & 0x7fffffu) | 0x800000u;
    const uint32_t rs = min(268u - 2u * e, 63u);
    emax = max(emax, e);
    return ((uint64_t)m * (uint64_t)m) >> rs;
}

// Wait for the previous pass to complete (its pool, state and scale visible),
// let the next pass's CTAs launch (they take SMs as this pass's CTAs leave
// and run their own prologue meanwhile), and return this pass's scale c.
// Every thread of the CTA calls.
// sub-vector of span s (spans are numbered sub-vector by sub-vector)
template <int NSUB>
__device__ __forceinline__ int tm_sub(int s, const int *sb)
{
    if constexpr (NSUB == 4)
        return (s >= sb[1]) + (s >= sb[2]) + (s >= sb[3]);
    else
        return s >= sb[1] ? 1 : 0;
}

} // namespace wl_tma
