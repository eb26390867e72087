// One pass of Wallace's generator by direct strided gather (Eq. 1 of Brent's
// RANN4 paper): thread t handles j = t, t + G, t + 2G, ... and reads
// g_i = x_i[(alpha_i j + gamma_i) mod N] straight from global memory.  As in
// the paper's vector loop (Section 7), no modulo is taken inside the loop:
// each index advances by alpha_i G mod N with one conditional subtraction.
// Works for every n, N and both pool precisions; the lane-tiled kernel
// (wl_tiled.cu) is the fast path for large binary32 pools.
#include "wl_common.cuh"
#include "wl_launch.h"

namespace {

template <int NSUB, typename T>
__global__ void __launch_bounds__(256) gather_kernel(WlPassArgs a)
{
    __shared__ uint64_t red[3 * 8];
    WlDevState *st = a.st;
    const T *__restrict__ src = (const T *)a.src;
    T *__restrict__ dst = (T *)a.dst;
    const int64_t N = a.N, Np = a.Np;
    constexpr bool f64 = sizeof(T) == 8;
    const T c = f64 ? (T)st->next.c64 : (T)st->next.c32;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t idx[NSUB], step[NSUB];
#pragma unroll
    for (int i = 0; i < NSUB; i++) {
        int64_t al = st->next.alpha[i], ga = st->next.gamma[i];
        idx[i] = (int64_t)(((uint64_t)al * (uint64_t)(j < N ? j : 0) + (uint64_t)ga) % (uint64_t)N);
        step[i] = (int64_t)(((uint64_t)al * (uint64_t)G) % (uint64_t)N);
    }
    T *out = (T *)a.out;
    const T mu = (T)a.mu, sigma = (T)a.sigma;
    const uint32_t signs = st->next.signs;
    const T rC = f64 ? (T)st->next.rc64 : (T)st->next.rc32;   // n = 2: rotation with the scale
    const T rS = f64 ? (T)st->next.rs64 : (T)st->next.rs32;
    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    for (; j < N; j += G) {
        T g[NSUB], y[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            g[i] = wl_sgn(src[i * Np + idx[i]], signs, i);
            idx[i] += step[i];
            if (idx[i] >= N)
                idx[i] -= N;
        }
        if constexpr (sizeof(T) == 8) {
            if constexpr (NSUB == 2)
                wl_xform2d(g, rC, rS, y);
            else if constexpr (NSUB == 4)
                wl_xform4d(g, c, y);
            else
                wl_xform8d(g, c, y);
        } else {
            if constexpr (NSUB == 2)
                wl_xform2(g, rC, rS, y);
            else if constexpr (NSUB == 4)
                wl_xform4(g, c, y);
            else
                wl_xform8(g, c, y);
        }
#pragma unroll
        for (int k = 0; k < NSUB; k++) {
            dst[k * Np + j] = y[k];
            int64_t q = k * N + j;
            if constexpr (sizeof(T) == 8) {
                uint64_t tl, th;
                wl_term64(y[k], tl, th, bad);
                wl_add128(lo, hi, tl, th);
                if (q >= a.w0 && q < a.w1)
                    out[q - a.w0] = __dadd_rn(mu, __dmul_rn(sigma, y[k]));
            } else {
                wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                if (q >= a.w0 && q < a.w1)
                    out[q - a.w0] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
            }
        }
    }
    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st) && threadIdx.x == 0) {
        double x = (double)__ldcg(&dst[wl_phys(a.nu - 1, N, Np)]);
        wl_finalise(st, a.n, N, a.nu, x, f64, WL_FIN_PASS);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) drain_kernel(const T *__restrict__ pool, int64_t N,
                                                    int64_t Np, int64_t pos, int64_t count,
                                                    T *__restrict__ out, double mu, double sigma)
{
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += G) {
        T y = pool[wl_phys(pos + k, N, Np)];
        if constexpr (sizeof(T) == 8)
            out[k] = __dadd_rn(mu, __dmul_rn(sigma, y));
        else
            out[k] = __fadd_rn((float)mu, __fmul_rn((float)sigma, y));
    }
}

} // namespace

cudaError_t wl_launch_gather(const WlPassArgs &a, int fp64, int sm_count, cudaStream_t stream)
{
    int64_t want = (a.N + 255) / 256;
    int64_t cap = (int64_t)sm_count * 8;
    int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    if (a.n == 2) {
        if (fp64)
            gather_kernel<2, double><<<grid, 256, 0, stream>>>(a);
        else
            gather_kernel<2, float><<<grid, 256, 0, stream>>>(a);
    } else if (a.n == 4) {
        if (fp64)
            gather_kernel<4, double><<<grid, 256, 0, stream>>>(a);
        else
            gather_kernel<4, float><<<grid, 256, 0, stream>>>(a);
    } else {
        if (fp64)
            gather_kernel<8, double><<<grid, 256, 0, stream>>>(a);
        else
            gather_kernel<8, float><<<grid, 256, 0, stream>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t wl_launch_drain(const void *pool, int fp64, int64_t N, int64_t Np, int64_t pos,
                            int64_t count, void *out, double mu, double sigma, int sm_count,
                            cudaStream_t stream)
{
    if (count <= 0)
        return cudaSuccess;
    int64_t want = (count + 255) / 256;
    int64_t cap = (int64_t)sm_count * 8;
    int grid = (int)(want < cap ? want : cap);
    if (fp64)
        drain_kernel<double><<<grid, 256, 0, stream>>>((const double *)pool, N, Np, pos, count,
                                                       (double *)out, mu, sigma);
    else
        drain_kernel<float><<<grid, 256, 0, stream>>>((const float *)pool, N, Np, pos, count,
                                                      (float *)out, mu, sigma);
    return cudaGetLastError();
}
