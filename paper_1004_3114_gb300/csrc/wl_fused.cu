// Many passes of Wallace's generator in one launch for a pool that fits in
// shared memory (Brent's RANN4 paper, Section 2: a pass is a few vector
// operations over the pool; here the pool never leaves the SM between
// passes, only the returned values go to global memory).
//
// One CTA owns the generator.  Per pass: thread 0 already holds the pass's
// strides, offsets and scale in the state (drawn by the previous
// finaliser); all threads gather from one shared buffer into the other
// (Eq. 1), accumulate the exact sum of squares, and write the returned prefix;
// thread 0 then runs the chi-squared rescale (Eq. 3) and drift check and draws
// the next parameters.  At the end the pool is written back to global memory.
#include <algorithm>

#include "wl_common.cuh"
#include "wl_launch.h"

#define FU_THREADS 512
#define FU_SMEM_MAX (220 * 1024)

namespace {

template <int NSUB, typename T>
__global__ void __launch_bounds__(FU_THREADS) fused_kernel(const T *gin, T *gout, int64_t N,
                                                          int64_t Np, WlDevState *st_g,
                                                          int64_t passes, int64_t R,
                                                          int64_t last_take, T *__restrict__ out,
                                                          double mu_d, double sigma_d)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ uint64_t red[3 * (FU_THREADS / 32)];
    __shared__ WlDevState sst;   // the state, on chip for the whole run
    wl_state_load(&sst, st_g);
    WlDevState *st = &sst;
    const int tid = threadIdx.x;
    const int nu = NSUB * (int)N;
    const double rnu = wl_rnu(nu);
    T *buf0 = (T *)fsm;
    T *buf1 = buf0 + nu;
    for (int q = tid; q < nu; q += blockDim.x) {
        int i = q / (int)N;
        buf0[q] = gin[(int64_t)i * Np + (q - i * (int)N)];
    }
    __syncthreads();   // the pool is on chip; each pass then ends with a barrier
    const T mu = (T)mu_d, sigma = (T)sigma_d;
    T *src = buf0, *dst = buf1;
    for (int64_t pass = 0; pass < passes; pass++) {
        // this pass's parameters, as the previous pass's end left them; thread
        // 0 records them as the most recent pass's (nothing writes `next`
        // until the end of the pass)
        if (tid == 0)
            st->last = st->next;
        int32_t s_alpha[NSUB], s_gamma[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            s_alpha[i] = st->next.alpha[i];
            s_gamma[i] = (int32_t)st->next.gamma[i];
        }
        T c, rC = (T)0, rS = (T)0;
        if constexpr (sizeof(T) == 8)
            c = st->next.c64;
        else
            c = st->next.c32;
        if constexpr (NSUB == 2) {
            // the scale folded into the rotation, as wl_fold_rotation does
            const double rc = __dmul_rn(st->next.c64, st->next.rcos);
            const double rs = __dmul_rn(st->next.c64, st->next.rsin);
            if constexpr (sizeof(T) == 8) {
                rC = rc;
                rS = rs;
            } else {
                rC = __double2float_rn(rc);
                rS = __double2float_rn(rs);
            }
        }
        const uint32_t signs = st->next.signs;
        const int take = (int)(pass + 1 < passes ? R : last_take);
        T *o = out + pass * R;
        // 32-bit index arithmetic: N <= 7040 here and alpha * blockDim < 2^32
        const uint32_t uN = (uint32_t)N, nth = blockDim.x;
        int idx[NSUB], stp[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            idx[i] = (int)(((uint32_t)s_alpha[i] * (uint32_t)(tid < (int)N ? tid : 0) + (uint32_t)s_gamma[i]) % uN);
            stp[i] = (int)(((uint32_t)s_alpha[i] * nth) % uN);
        }
        uint64_t lo = 0, hi = 0;
        uint32_t bad = 0;
        for (int j = tid; j < (int)N; j += (int)nth) {
            T g[NSUB], y[NSUB];
#pragma unroll
            for (int i = 0; i < NSUB; i++) {
                g[i] = wl_sgn(src[i * (int)N + idx[i]], signs, i);
                idx[i] += stp[i];
                if (idx[i] >= (int)N)
                    idx[i] -= (int)N;
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
                int q = k * (int)N + j;
                dst[q] = y[k];
                if constexpr (sizeof(T) == 8) {
                    uint64_t tl, th;
                    wl_term64(y[k], tl, th, bad);
                    wl_add128(lo, hi, tl, th);
                    if (q < take)
                        o[q] = __dadd_rn(mu, __dmul_rn(sigma, y[k]));
                } else {
                    wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                    if (q < take)
                        o[q] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
                }
            }
        }
        const T *xp = &dst[nu - 1];
        wl_end_pass_cta(st, NSUB, N, (int64_t)nu, rnu, lo, hi, bad, red, [xp]() { return (double)*xp; },
                        st->msigns, sizeof(T) == 8);
        T *t = src;
        src = dst;
        dst = t;
    }
    if (NSUB == 2 && tid == 0)
        wl_fold_rotation(st);
    for (int q = tid; q < nu; q += blockDim.x) {
        int i = q / (int)N;
        gout[(int64_t)i * Np + (q - i * (int)N)] = src[q];
    }
    wl_state_store(st_g, &sst);
}

template <int NSUB, typename T>
cudaError_t launch_one(void *pin, void *pout, int64_t N, int64_t Np, WlDevState *st, int64_t passes,
                       int64_t R, int64_t last_take, void *out, double mu, double sigma,
                       cudaStream_t stream)
{
    static bool configured = false;
    const size_t smem = 2 * sizeof(T) * (size_t)NSUB * (size_t)N;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(fused_kernel<NSUB, T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             FU_SMEM_MAX);
        if (e != cudaSuccess)
            return e;
        configured = true;
    }
    // one thread per tuple up to FU_THREADS (at least four warps: the
    // finaliser's chains take three): fewer idle threads at each barrier
    const int threads = (int)std::min<int64_t>(FU_THREADS, std::max<int64_t>(128, (N + 31) / 32 * 32));
    fused_kernel<NSUB, T><<<1, threads, smem, stream>>>((const T *)pin, (T *)pout, N, Np, st,
                                                          passes, R, last_take, (T *)out, mu,
                                                          sigma);
    return cudaGetLastError();
}

} // namespace

bool wl_fused_supported(int n, int64_t N, int fp64, int64_t *smem_bytes)
{
    int64_t bytes = 2 * (fp64 ? 8 : 4) * (int64_t)n * N;
    if (smem_bytes)
        *smem_bytes = bytes;
    return (n == 2 || n == 4 || n == 8) && N >= 4 && bytes <= FU_SMEM_MAX;
}

cudaError_t wl_launch_fused(void *pool_cur, void *pool_other, int fp64, int n, int64_t N,
                            int64_t Np, WlDevState *st, int64_t passes, int64_t R,
                            int64_t last_take, void *out, double mu, double sigma,
                            cudaStream_t stream)
{
    (void)pool_other;
    if (passes <= 0)
        return cudaSuccess;
    if (n == 2)
        return fp64 ? launch_one<2, double>(pool_cur, pool_cur, N, Np, st, passes, R, last_take,
                                            out, mu, sigma, stream)
                    : launch_one<2, float>(pool_cur, pool_cur, N, Np, st, passes, R, last_take,
                                           out, mu, sigma, stream);
    if (n == 4)
        return fp64 ? launch_one<4, double>(pool_cur, pool_cur, N, Np, st, passes, R, last_take,
                                            out, mu, sigma, stream)
                    : launch_one<4, float>(pool_cur, pool_cur, N, Np, st, passes, R, last_take,
                                           out, mu, sigma, stream);
    return fp64 ? launch_one<8, double>(pool_cur, pool_cur, N, Np, st, passes, R, last_take, out,
                                        mu, sigma, stream)
                : launch_one<8, float>(pool_cur, pool_cur, N, Np, st, passes, R, last_take, out,
                                       mu, sigma, stream);
}
