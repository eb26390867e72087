// A CTA-local form of the bulk-copy (TMA) pass: one CTA of TM_THREADS threads
// runs every pass of one n = 4 generator itself (the batched generators of
// wl_batch.cu), with the same lane-tiled geometry and warp-specialised stage
// ring as the grid-wide kernel (wl_tiled_tma.cu) -- 4 producer warps issue
// one bulk copy per span into TM_STAGES shared-memory stages, 15 consumer
// warps own 3 lanes each -- but over all tiles of the pool in order, with the
// sum of squares and the chi-squared rescale (Eq. 3 of Brent's RANN4 paper)
// done by the CTA itself, so no CTA waits for another.
//
// The ring's mbarriers are initialised once per CTA and `it` counts the
// stage uses so far (the same in every thread), so the phase parities stay
// right across passes and generators.  Every wait is bounded; after a
// timeout the CTA records WALLACE_ETIMEOUT in the generator's state, waits
// (bounded) for its copies in flight and runs no more bulk-copy passes.
#pragma once

#include "wl_run_body.cuh"
#include "wl_tma_common.cuh"

struct WlTmaRing {
    uint64_t *full, *empty;    // TM_STAGES mbarriers each, in shared memory
    int it;                    // stage uses so far
    volatile int *abort_flag;  // shared: a wait timed out in this CTA
};

// Once per CTA, by every thread.
__device__ inline void wl_tma_ring_init(WlTmaRing &r)
{
    using namespace wl_tma;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TM_STAGES; s++) {
            mbar_init(smem_u32(&r.full[s]), 32 * TM_PROD_WARPS);
            mbar_init(smem_u32(&r.empty[s]), TM_CONS_WARPS);
        }
        *r.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    r.it = 0;
}

// Lanes of the tiled geometry for these strides (lcm, all dividing 45), or 0
// when a stride does not divide 45 (the coprimality fallback).
__device__ __forceinline__ int wl_tma_lanes45(const int32_t *alpha)
{
    int e3 = 0, e5 = 0;
    for (int i = 0; i < 4; i++) {
        const int al = alpha[i];
        if (al != 3 && al != 5 && al != 9 && al != 15 && al != 45)
            return 0;
        if (al == 3 || al == 15)
            e3 = max(e3, 1);
        if (al == 9 || al == 45)
            e3 = 2;
        if (al == 5 || al == 15 || al == 45)
            e5 = 1;
    }
    return (e3 == 2 ? 9 : (e3 == 1 ? 3 : 1)) * (e5 ? 5 : 1);
}

// One pass src -> dst of an n = 4 pool (N % 4 == 0, N >= TM_MIN_N) whose
// strides have lcm L <= 45.  Every thread of the CTA calls; the terms of its
// values are added to (lo, hi) and its bad-value flag to `bad`.  The pass's
// returned values [0, w1) go to o (o may be null when w1 == 0).
__device__ inline void wl_tma_pass_cta(const float *src, float *dst, int64_t N, int64_t Np, int L,
                                       const int32_t *alpha, const int64_t *gam, float c, float *o,
                                       int64_t w1, float mu, float sigma, float *smem, WlTmaRing &ring,
                                       WlDevState *st, uint64_t &lo, uint64_t &hi, uint32_t &bad)
{
    using namespace wl_tma;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int m[4], sb[5];
    sb[0] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        m[i] = tm_divc(L, alpha[i]);
        sb[i + 1] = sb[i] + m[i];
    }
    const int nspans = sb[4];
    const int T = tm_divc(TM_ETARGET, L);
    int SL[4], slot0[4];
    slot0[0] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        SL[i] = (alpha[i] * T + 8 + 3) & ~3;   // 16-byte aligned slots; wrap copies need +6
        if (i < 3)
            slot0[i + 1] = slot0[i] + m[i] * SL[i];
    }
    float *stage0 = smem;
    int *common = (int *)(smem + TM_STAGES * tm_stage_words());
    int *J = common;
    int *lanebase = J + (TM_LMAX2 + 1);
    int *spanC = lanebase + 4 * TM_LMAX;

    // the previous pass's readers of the tables are done
    __syncthreads();
    const int N32 = (int)N;
    for (int l = tid; l <= L; l += TM_THREADS) {
        const int qN = tm_divc(N32, L), rN = N32 - qN * L;
        J[l] = l * qN + tm_divc(l * rN + L - 1, L);
    }
    for (int s = tid; s < nspans; s += TM_THREADS) {
        const int i = tm_sub<4>(s, sb);
        const int p = s - sb[i], mi = m[i];
        const int qN = tm_divc(N32, mi), rN = N32 - qN * mi;
        spanC[s] = p * qN + tm_divc(p * rN + mi - 1, mi);
    }
    __syncthreads();
    for (int e = tid; e < 4 * L; e += TM_THREADS) {
        int i = tm_divc(e, L), l = e - i * L;
        int w = tm_divc(l, m[i]), p = l - w * m[i];
        int64_t r = (int64_t)alpha[i] * J[l] - (int64_t)w * N - spanC[sb[i] + p];
        lanebase[i * TM_LMAX + l] = ((slot0[i] + p * SL[i] + (int)r) << 5) | (sb[i] + p);
    }
    __syncthreads();
    const int maxlen = tm_divc(N32 + L - 1, L);
    const int ntiles = (maxlen + T - 1) / T;
    const int it0 = ring.it;

    if (warp >= TM_CONS_WARPS) {
        // ---------------- producer warps ----------------
        const int sp = (warp - TM_CONS_WARPS) + TM_PROD_WARPS * lane;
        const bool owner = sp < nspans;
        int sp_i = 0, sp_alpha = 0;
        int64_t sp_gam = 0, sp_C = 0;
        uint32_t sp_doff = 0;
        const float *sp_row = src;
        if (owner) {
            sp_i = tm_sub<4>(sp, sb);
            const int sp_p = sp - sb[sp_i];
            sp_alpha = alpha[sp_i];
            sp_gam = gam[sp_i];
            sp_C = spanC[sp];
            sp_doff = 4u * (uint32_t)(slot0[sp_i] + sp_p * SL[sp_i]);
            sp_row = src + (int64_t)sp_i * Np;
        }
        const uint32_t stage_base = smem_u32(stage0);
        int issued_last = -1;   // last ring use this thread issued
        for (int tile = 0; tile < ntiles; tile++) {
            const int g = it0 + tile, s = g % TM_STAGES, u = g / TM_STAGES;
            if (*ring.abort_flag)
                break;
            if (u > 0 && !mbar_wait(smem_u32(&ring.empty[s]), (uint32_t)((u - 1) & 1))) {
                *ring.abort_flag = 1;
                atomicOr(&st->status, WL_ETIMEOUT);
                break;
            }
            const int t0 = tile * T;
            const int Tt = min(T, maxlen - t0);
            int *lead = (int *)(stage0 + s * tm_stage_words() + tm_stage_data_words());
            const uint32_t full = smem_u32(&ring.full[s]);
            const uint32_t d = stage_base + 4u * (uint32_t)(s * tm_stage_words()) + sp_doff;
            int64_t addr = 0;
            int len = 0, as = 0;
            uint32_t bytes = 0;
            bool wrap = false;
            if (owner) {
                addr = sp_C + (int64_t)sp_alpha * t0 + sp_gam;   // < 3N
                if (addr >= N)
                    addr -= N;
                if (addr >= N)
                    addr -= N;
                len = sp_alpha * Tt;
                as = (int)addr & ~3;
                lead[sp] = (int)addr - as;
                wrap = addr + len > N;
                bytes = wrap ? 4u * (uint32_t)((int)N - as) + 4u * (uint32_t)(((int)(addr + len - N) + 3) & ~3)
                             : 16u * (uint32_t)(((int)addr - as + len + 3) >> 2);
            }
            uint32_t total = bytes;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                total += __shfl_xor_sync(0xffffffffu, total, off);
            if (lane == 0)
                mbar_expect_tx(full, total);
            __syncwarp();
            if (owner) {
                if (!wrap) {
                    bulk_g2s(d, sp_row + as, bytes, full);
                } else {
                    const int e2 = ((int)(addr + len - N) + 3) & ~3;
                    bulk_g2s(d, sp_row + as, 4u * (uint32_t)((int)N - as), full);
                    bulk_g2s(d + 4u * (uint32_t)((int)N - as), sp_row, 4u * (uint32_t)e2, full);
                }
            }
            mbar_arrive(full);
            issued_last = g;
        }
        if (*ring.abort_flag) {
            // copies still in flight must land before the CTA moves on
            for (int g = max(it0, issued_last - TM_STAGES + 1); g <= issued_last; g++)
                if (!mbar_wait(smem_u32(&ring.full[g % TM_STAGES]), (uint32_t)((g / TM_STAGES) & 1)))
                    atomicOr(&st->status, WL_ETIMEOUT);
        }
    } else {
        // ---------------- consumer warps ----------------
        float *dstk[4], *outk[4];
        bool ret[4];   // sub-vector k lies wholly in the returned prefix
#pragma unroll
        for (int k = 0; k < 4; k++) {
            dstk[k] = dst + k * Np;
            ret[k] = (int64_t)(k + 1) * N <= w1;
            outk[k] = ret[k] ? o + k * N : o;
        }
        uint32_t emax = 0;
        for (int tile = 0; tile < ntiles; tile++) {
            const int g = it0 + tile, s = g % TM_STAGES, u = g / TM_STAGES;
            if (*ring.abort_flag)
                break;
            if (!mbar_wait(smem_u32(&ring.full[s]), (uint32_t)(u & 1))) {
                *ring.abort_flag = 1;
                atomicOr(&st->status, WL_ETIMEOUT);
                break;
            }
            const int t0 = tile * T;
            const int Tt = min(T, maxlen - t0);
            const float *sdata = stage0 + s * tm_stage_words();
            const int *lead = (const int *)(sdata + tm_stage_data_words());
            uint64_t tl = 0;   // this tile's terms: at most 24 per thread, each below 2^48
            for (int l = warp; l < L; l += TM_CONS_WARPS) {
                const int jl = J[l];
                const int tmax = min(Tt, J[l + 1] - jl - t0);
                const float *gp[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int lb = lanebase[i * TM_LMAX + l];
                    gp[i] = sdata + (lb >> 5) + lead[lb & 31];
                }
                const int64_t jb = (int64_t)jl + t0;
                for (int t = lane; t < tmax; t += 64) {
                    const bool v2 = t + 32 < tmax;
                    float gv[4], h[4], y[4], z[4];
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        gv[i] = gp[i][alpha[i] * t];
                        h[i] = v2 ? gp[i][alpha[i] * (t + 32)] : 0.f;
                    }
                    wl_xform4(gv, c, y);
                    wl_xform4(h, c, z);
                    const int64_t j = jb + t;
#pragma unroll
                    for (int kk = 0; kk < 4; kk++) {
                        dstk[kk][j] = y[kk];
                        if (v2) dstk[kk][j + 32] = z[kk];
                        tl += term32(y[kk], emax);
                        if (v2) tl += term32(z[kk], emax);
                        if (ret[kk]) {
                            outk[kk][j] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                            if (v2) outk[kk][j + 32] = __fadd_rn(mu, __fmul_rn(sigma, z[kk]));
                        } else {
                            const int64_t q = kk * N + j;
                            if (q < w1)
                                o[q] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                            if (v2 && q + 32 < w1)
                                o[q + 32] = __fadd_rn(mu, __fmul_rn(sigma, z[kk]));
                        }
                    }
                }
            }
            lo += tl;
            hi += lo < tl ? 1ull : 0ull;
            __syncwarp();
            if (lane == 0)
                mbar_arrive(smem_u32(&ring.empty[s]));
        }
        bad |= emax >= 135u ? 1u : 0u;
        // the next pass reads this pool with bulk copies (the async proxy)
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
    }
    ring.it = it0 + ntiles;
}

// All passes of the spec (n = 4, N % 4 == 0, N >= TM_MIN_N) from global
// memory through the bulk-copy pass; a pass whose strides do not all divide
// 45 takes the plain gather.  Returns the index of the buffer holding the
// final pool.  s_prm: at least 9 words of shared memory.
__device__ inline int wl_run_tma(const WlRunSpec &d, float *smem, uint64_t *red, int32_t *s_prm,
                                 WlTmaRing &ring)
{
    const int tid = threadIdx.x;
    const int64_t N = d.N, nu = 4 * N;
    const double rnu = wl_rnu(nu);
    int cur = d.cur;
    for (int64_t p = 0; p < d.passes; p++) {
        __syncthreads();   // the previous pass's finaliser has written the parameters
        if (tid < 4) {
            s_prm[tid] = d.st->next.alpha[tid];
            s_prm[4 + tid] = (int32_t)d.st->next.gamma[tid];
        } else if (tid == 4) {
            s_prm[8] = __float_as_int(d.st->next.c32);
        }
        __syncthreads();
        int32_t alpha[4];
        int64_t gam[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            alpha[i] = s_prm[i];
            gam[i] = s_prm[4 + i];
        }
        const float c = __int_as_float(s_prm[8]);
        const float *src = d.buf[cur];
        float *dst = d.buf[1 - cur];
        float *o = d.out ? d.out + p * d.R : nullptr;
        const int64_t w1 = o ? (p + 1 < d.passes ? d.R : d.last_take) : 0;
        uint64_t lo = 0, hi = 0;
        uint32_t bad = 0;
        const int L = wl_tma_lanes45(alpha);
        if (L > 0 && !*ring.abort_flag) {
            wl_tma_pass_cta(src, dst, N, d.Np, L, alpha, gam, c, o, w1, d.mu, d.sigma, smem, ring, d.st,
                            lo, hi, bad);
        } else {
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
            job.out = o;
            job.w0 = 0;
            job.w1 = w1;
            job.mu = d.mu;
            job.sigma = d.sigma;
            wl_gather4_range(job, tid, blockDim.x, lo, hi, bad);
            // the next pass may read this pool with bulk copies
            asm volatile("fence.proxy.async.global;\n" ::: "memory");
        }
        wl_cta_reduce_to_state(lo, hi, bad, d.st, red);
        __syncthreads();
        const float *xp = &dst[wl_phys(nu - 1, N, d.Np)];
        wl_finalise_par(d.st, 4, N, nu, rnu, [xp]() { return (double)__ldcg(xp); }, d.st->msigns, false);
        cur = 1 - cur;
    }
    return cur;
}
