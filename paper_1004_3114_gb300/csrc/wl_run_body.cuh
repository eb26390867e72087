// Per-CTA runners that advance ONE generator by several passes, shared by
// the batched kernel (wl_batch.cu) and the serving kernel (wl_serve.cu).
// A CTA owns the generator for the whole call, so the sum of squares and the
// chi-squared rescale (Eq. 3 of Brent's RANN4 paper) are CTA-local.
#pragma once

#include "wl_tiled_body.cuh"

// What one CTA does for one generator.
struct WlRunSpec {
    float *buf[2];       // pool buffers; the pool is in buf[cur]
    int cur;
    WlDevState *st;
    int64_t N, Np, R;
    int n;
    int64_t passes;
    float *out;          // pass p writes its first take values to out + p * R (may be null)
    int64_t last_take;   // values the last pass returns (the others return R)
    float mu, sigma;
    int etarget;         // lane-times per tile of the tiled gather
};

// plain strided gather of j in [j0, j_end) (j_end < 0: N), thread t taking
// j0 + t, j0 + t + blockDim, ...
// signs: the pass's sign pattern (bit i negates g_i; 0 for the fixed matrix)
template <int NSUB>
__device__ void wl_gather_range_n(const float *src, float *dst, int64_t N, int64_t Np,
                                  const int32_t *alpha, const int64_t *gam, float c, float *out,
                                  int64_t w1, float mu, float sigma, uint64_t &lo, uint64_t &hi,
                                  uint32_t &bad, int64_t j0 = 0, int64_t j_end = -1, uint32_t signs = 0)
{
    const int64_t G = blockDim.x;
    int64_t j = j0 + threadIdx.x;
    const int64_t jmax = j_end < 0 ? N : j_end;
    int64_t idx[NSUB], stp[NSUB];
#pragma unroll
    for (int i = 0; i < NSUB; i++) {
        idx[i] = (int64_t)(((uint64_t)alpha[i] * (uint64_t)(j < N ? j : 0) + (uint64_t)gam[i]) % (uint64_t)N);
        stp[i] = (int64_t)(((uint64_t)alpha[i] * (uint64_t)G) % (uint64_t)N);
    }
    for (; j < jmax; j += G) {
        float g[NSUB], y[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            g[i] = wl_sgn(src[i * Np + idx[i]], signs, i);
            idx[i] += stp[i];
            if (idx[i] >= N)
                idx[i] -= N;
        }
        if constexpr (NSUB == 4)
            wl_xform4(g, c, y);
        else
            wl_xform8(g, c, y);
#pragma unroll
        for (int k = 0; k < NSUB; k++) {
            dst[k * Np + j] = y[k];
            wl_add128(lo, hi, wl_term32(y[k], bad), 0);
            const int64_t q = k * N + j;
            if (q < w1)
                out[q] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
        }
    }
}

// All passes with the pool in shared memory (2 n N floats of `sm`); the pool
// is written back to buf[cur] at the end.
// SG (here and below): the generator draws a sign pattern each pass (matrix
// A D_k); without it the runner carries no sign code.
template <int NSUB, bool SG>
__device__ void wl_run_fused(const WlRunSpec &d, float *sm, uint64_t *red)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    const int N = (int)d.N, nu = NSUB * N;
    const double rnu = wl_rnu(nu);
    float *src = sm, *dst = sm + nu;
    const float *g0 = d.buf[d.cur];
    for (int q = tid; q < nu; q += nth) {
        int i = q / N;
        src[q] = g0[(int64_t)i * d.Np + (q - i * N)];
    }
    __syncthreads();   // the pool is on chip; each pass then ends with a barrier
    WlDevState *st = d.st;   // the CTA's shared-memory copy of the state
    for (int64_t p = 0; p < d.passes; p++) {
        // this pass's parameters, as the previous pass's end left them; thread
        // 0 records them as the most recent pass's
        if (tid == 0)
            st->last = st->next;
        const float c = st->next.c32;
        const uint32_t signs = SG ? st->next.signs : 0u;   // the pass's sign pattern (matrix A D_k)
        // 32-bit index arithmetic: a pool in shared memory has N < 2^13 and
        // alpha * blockDim < 2^32
        int32_t al[NSUB];
        int idx[NSUB], stp[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            al[i] = st->next.alpha[i];
            idx[i] = (int)(((uint32_t)al[i] * (uint32_t)(tid < N ? tid : 0) + (uint32_t)st->next.gamma[i]) %
                           (uint32_t)N);
            stp[i] = (int)(((uint32_t)al[i] * (uint32_t)nth) % (uint32_t)N);
        }
        float *o = d.out ? d.out + p * d.R : nullptr;
        const int w1 = o ? (int)(p + 1 < d.passes ? d.R : d.last_take) : 0;
        uint64_t lo = 0, hi = 0;
        uint32_t bad = 0;
        for (int j = tid; j < N; j += nth) {
            float g[NSUB], y[NSUB];
#pragma unroll
            for (int i = 0; i < NSUB; i++) {
                g[i] = SG ? wl_sgn(src[i * N + idx[i]], signs, i) : src[i * N + idx[i]];
                idx[i] += stp[i];
                if (idx[i] >= N)
                    idx[i] -= N;
            }
            if constexpr (NSUB == 4)
                wl_xform4(g, c, y);
            else
                wl_xform8(g, c, y);
#pragma unroll
            for (int k = 0; k < NSUB; k++) {
                const int q = k * N + j;
                dst[q] = y[k];
                wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                if (q < w1)
                    o[q] = __fadd_rn(d.mu, __fmul_rn(d.sigma, y[k]));
            }
        }
        const float *xp = &dst[nu - 1];
        wl_end_pass_cta(st, NSUB, N, nu, rnu, lo, hi, bad, red, [xp]() { return (double)*xp; }, st->msigns,
                        false);
        float *t = src;
        src = dst;
        dst = t;
    }
    float *g1 = d.buf[d.cur];
    for (int q = tid; q < nu; q += nth) {
        int i = q / N;
        g1[(int64_t)i * d.Np + (q - i * N)] = src[q];
    }
}

// All passes from global memory, alternating buf[cur] and buf[1 - cur];
// returns the index of the buffer holding the final pool.
template <int NSUB, bool SG>
__device__ int wl_run_global(const WlRunSpec &d, float *sm, uint64_t *red)
{
    const int tid = threadIdx.x;
    const int64_t N = d.N, nu = NSUB * N;
    const double rnu = wl_rnu(nu);
    int cur = d.cur;
    WlDevState *st = d.st;   // the CTA's shared-memory copy of the state
    for (int64_t p = 0; p < d.passes; p++) {
        // parameters as the previous pass's end (a barrier) left them
        if (tid == 0)
            st->last = st->next;
        int32_t alpha[NSUB];
        int64_t gam[NSUB];
#pragma unroll
        for (int i = 0; i < NSUB; i++) {
            alpha[i] = st->next.alpha[i];
            gam[i] = st->next.gamma[i];
        }
        const float c = st->next.c32;
        const float *src = d.buf[cur];
        float *dst = d.buf[1 - cur];
        float *o = d.out ? d.out + p * d.R : nullptr;
        const int64_t w1 = o ? (p + 1 < d.passes ? d.R : d.last_take) : 0;
        uint64_t lo = 0, hi = 0;
        uint32_t bad = 0;
        if constexpr (NSUB == 4) {
            WlTileJob job;
            job.src = src;
            job.dst = dst;
            job.N = N;
            job.Np = d.Np;
            for (int i = 0; i < 4; i++) {
                job.alpha[i] = alpha[i];
                job.gam[i] = gam[i];
            }
            job.c = c;
            job.signs = SG ? st->next.signs : 0u;
            job.out = o;
            job.w0 = 0;
            job.w1 = w1;
            job.mu = d.mu;
            job.sigma = d.sigma;
            const int L = wl_lcm4(job.alpha);
            if (wl_tiled_ok(L, N))
                wl_tiled4_tiles(job, L, 0, 1, d.etarget, sm, lo, hi, bad);
            else
                wl_gather4_range(job, tid, blockDim.x, lo, hi, bad);
        } else {
            wl_gather_range_n<NSUB>(src, dst, N, d.Np, alpha, gam, c, o, w1, d.mu, d.sigma, lo, hi,
                                    bad, 0, -1, SG ? st->next.signs : 0u);
        }
        const float *xp = &dst[wl_last_phys(NSUB, N, d.Np)];
        wl_end_pass_cta(st, NSUB, N, nu, rnu, lo, hi, bad, red, [xp]() { return (double)__ldcg(xp); },
                        st->msigns, false);
        cur = 1 - cur;
    }
    return cur;
}

// Runs the spec on the fused path when the pool fits the shared memory the
// caller has (smem_values floats) and n N <= fused_max; returns the final
// buffer index (unchanged for the fused path, which writes back in place).
template <bool SG = false>
__device__ inline int wl_run_spec(const WlRunSpec &d, int64_t fused_max, int64_t smem_values, float *sm,
                                  uint64_t *red)
{
    const int64_t nu = (int64_t)d.n * d.N;
    if (nu <= fused_max && 2 * nu <= smem_values) {
        if (d.n == 4)
            wl_run_fused<4, SG>(d, sm, red);
        else
            wl_run_fused<8, SG>(d, sm, red);
        return d.cur;
    }
    return d.n == 4 ? wl_run_global<4, SG>(d, sm, red) : wl_run_global<8, SG>(d, sm, red);
}

// Whether wl_run_spec takes the fused path (the host uses the same rule to
// know where the pool ends up).
__host__ __device__ inline bool wl_run_is_fused(int n, int64_t N, int64_t fused_max, int64_t smem_values)
{
    const int64_t nu = (int64_t)n * N;
    return nu <= fused_max && 2 * nu <= smem_values;
}
