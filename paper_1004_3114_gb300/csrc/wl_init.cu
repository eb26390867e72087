// Initial pool of a Wallace generator: Box-Muller pairs from the uniform
// source (Sections 5 and 8 of Brent's RANN4 paper), its exact sum of squares,
// and the first chi-squared target (Eq. 3) -- one launch.  The Box-Muller
// arithmetic (binary64, project-written series) is in wl_bm.cuh.
#include "wl_bm.cuh"
#include "wl_common.cuh"
#include "wl_launch.h"

namespace {

using wl_bm::box_muller;

// kind = WL_FIN_INIT: the pool of a new generator, from uniforms [0, nu).
// kind = WL_FIN_RESTART: restart r refills the current pool from uniforms
// [r 2^40, r 2^40 + nu) of the same sequence (Section 5, restarting).
template <typename T>
__global__ void __launch_bounds__(256) init_kernel(T *pool, int n, int64_t N, int64_t Np,
                                                   int64_t nu, uint32_t seed, uint32_t stream,
                                                   WlDevState *st, int opts, int kind,
                                                   uint64_t restart)
{
    __shared__ uint64_t red[3 * 8];
    const uint64_t s0 = wl_seed_mix(seed, stream);
    const uint64_t base = wl_lcg_jump(s0, restart << 40);
    const int64_t npairs = nu / 2;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // map for 2G steps, to hop from pair p to pair p + G
    const uint64_t one = wl_lcg_jump(0, 2 * (uint64_t)G);         // C_{2G}
    const uint64_t AG = wl_lcg_jump(1, 2 * (uint64_t)G) - one;     // A_{2G}
    uint64_t s = wl_lcg_jump(base, 2 * (uint64_t)p);
    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    for (; p < npairs; p += G) {
        uint64_t t = s;
        uint32_t u1 = wl_lcg_step(t);
        uint32_t u2 = wl_lcg_step(t);
        float a, b;
        box_muller(u1, u2, a, b);
        int64_t q = 2 * p;
        pool[wl_phys(q, N, Np)] = (T)a;
        pool[wl_phys(q + 1, N, Np)] = (T)b;
        if (sizeof(T) == 4) {
            wl_add128(lo, hi, wl_term32(a, bad), 0);
            wl_add128(lo, hi, wl_term32(b, bad), 0);
        } else {
            uint64_t tl, th;
            wl_term64((double)a, tl, th, bad);
            wl_add128(lo, hi, tl, th);
            wl_term64((double)b, tl, th, bad);
            wl_add128(lo, hi, tl, th);
        }
        s = AG * s + one;
    }
    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st) && threadIdx.x == 0) {
        if (kind == WL_FIN_INIT) {
            st->lcg = wl_lcg_jump(s0, (uint64_t)nu);
            st->chi = opts & 1;
            st->msigns = (opts >> 1) & 1;
        }
        double x = (double)__ldcg(&pool[wl_phys(nu - 1, N, Np)]);
        wl_finalise(st, n, N, nu, x, sizeof(T) == 8, kind);
    }
}

} // namespace

cudaError_t wl_launch_init(void *pool, int fp64, int n, int64_t N, int64_t Np, uint32_t seed,
                           uint32_t stream_id, WlDevState *st, int sm_count, cudaStream_t stream,
                           int opts)
{
    int64_t nu = (int64_t)n * N;
    int64_t npairs = nu / 2;
    int64_t want = (npairs + 255) / 256;
    int64_t cap = (int64_t)sm_count * 8;
    int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    if (fp64)
        init_kernel<double><<<grid, 256, 0, stream>>>((double *)pool, n, N, Np, nu, seed,
                                                      stream_id, st, opts, WL_FIN_INIT, 0);
    else
        init_kernel<float><<<grid, 256, 0, stream>>>((float *)pool, n, N, Np, nu, seed,
                                                     stream_id, st, opts, WL_FIN_INIT, 0);
    return cudaGetLastError();
}

cudaError_t wl_launch_restart(void *pool, int fp64, int n, int64_t N, int64_t Np, uint32_t seed,
                              uint32_t stream_id, int64_t r, WlDevState *st, int sm_count,
                              cudaStream_t stream)
{
    int64_t nu = (int64_t)n * N;
    int64_t npairs = nu / 2;
    int64_t want = (npairs + 255) / 256;
    int64_t cap = (int64_t)sm_count * 8;
    int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    if (fp64)
        init_kernel<double><<<grid, 256, 0, stream>>>((double *)pool, n, N, Np, nu, seed,
                                                      stream_id, st, 0, WL_FIN_RESTART, (uint64_t)r);
    else
        init_kernel<float><<<grid, 256, 0, stream>>>((float *)pool, n, N, Np, nu, seed,
                                                     stream_id, st, 0, WL_FIN_RESTART, (uint64_t)r);
    return cudaGetLastError();
}
