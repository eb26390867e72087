// A CTA-local form of the bulk-copy (TMA) pass: one CTA of TM_THREADS threads
// runs every pass of one n = 4 generator itself (the batched generators of
// wl_batch.cu), with the same lane-tiled geometry and warp-specialised stage
// ring as the grid-wide kernel (wl_tiled_tma.cu) -- 4 producer warps issue
// one bulk copy per span into TR_STAGES shared-memory stages, 15 consumer
// warps own whole lanes (T >= TR_LANE_MIN_T) or take (lane, time) pairs --
// but over all tiles of the pool in order, for any N >= TR_MIN_N and lane
// counts up to TR_LMAX, with the sum of squares and the chi-squared rescale
// (Eq. 3 of Brent's RANN4 paper) done by the CTA itself (wl_end_pass_cta),
// so no CTA waits for another.
//
// The ring's mbarriers are initialised once per CTA and `it` counts the
// stage uses so far (the same in every thread), so the phase parities stay
// right across passes and generators.  Every wait is bounded; after a
// timeout the CTA records WALLACE_ETIMEOUT in the generator's state, waits
// (bounded) for its copies in flight and runs no more bulk-copy passes.
#pragma once

#include <type_traits>

#include "wl_run_body.cuh"
#include "wl_tma_common.cuh"

// Ring shape: TR_STAGES stages of up to TR_ETARGET values per sub-vector.  Longer
// tiles than the grid-wide kernel's (2880 in three stages) give lane counts
// above 45 lanes of at least 24 values (L <= 220), hence whole-lane
// consumers and fewer, longer bulk copies; the whole shared-memory block
// (about 192 KiB) still leaves the L1 share the plain-gather pools rely on.
#ifndef TR_STAGES
#define TR_STAGES 2
#endif
static_assert(TR_STAGES >= 2 && TR_STAGES <= 4, "the runner's ring rotates 2 to 4 stages (or uses them as one)");
#ifndef TR_ETARGET
#define TR_ETARGET 5280  /* values per sub-vector per tile: L T <= this */
#endif
#ifndef TR_LANE_MIN_T
#define TR_LANE_MIN_T 24 /* consumers own whole lanes when T is at least this */
#endif
#ifndef TR_ONE_STAGE_L
#define TR_ONE_STAGE_L 63 /* from this many lanes on, the stages form one stage of twice T */
#endif

struct WlTmaRing {
    uint64_t *full, *empty;    // TR_STAGES mbarriers each, in shared memory
    int uses[TR_STAGES];       // completed uses of each stage's barriers (the same in every thread)
    volatile int *abort_flag;  // shared: a wait timed out in this CTA
};

// Once per CTA, by every thread.
__device__ inline void wl_tma_ring_init(WlTmaRing &r)
{
    using namespace wl_tma;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TR_STAGES; s++) {
            mbar_init(smem_u32(&r.full[s]), 32 * TM_PROD_WARPS);
            mbar_init(smem_u32(&r.empty[s]), TM_CONS_WARPS);
        }
        *r.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    for (int s = 0; s < TR_STAGES; s++)
        r.uses[s] = 0;
}

// Geometry limits of the runner.  The strides of a pass have lcm L dividing
// p^2 q (p < q the smallest odd primes not dividing N): 45, 63, 99, 175, 275
// or 539 unless 105 or 165 divides N.  With T = TR_ETARGET / L lane times a
// tile still holds about TR_ETARGET values per sub-vector; the spans per tile
// are sum_i L / alpha_i <= 77 + 49 + 11 + 7 for L = 539.
#define TR_LMAX 539
/* from this many lanes on (the 539-lane stride sets) a tile's store runs are
   19 values: the returned values are then copied from the new pool after the
   pass instead of being stored beside it */
#define TR_RETURN_COPY_L 539
#define TR_MAXSPANS 144
#define TR_SPAN_PAD 12   /* slot words per span beyond alpha T: 3 lead + 3 wrap shift, rounded to 4 */

namespace wl_tma {

// stage: span data, then per span its lead and shift, then its wrap threshold
__host__ __device__ constexpr int tr_stage_data_words() { return 4 * TR_ETARGET + TR_SPAN_PAD * TR_MAXSPANS; }
__host__ __device__ constexpr int tr_stage_words() { return tr_stage_data_words() + 2 * TR_MAXSPANS; }
// common area: J[L + 1], lane table (4 rows of TR_LMAX), span starts
__host__ __device__ constexpr int tr_common_words() { return (TR_LMAX + 1) + 4 * TR_LMAX + TR_MAXSPANS; }
__host__ __device__ constexpr size_t tr_smem_bytes()
{
    return sizeof(float) * (size_t)(TR_STAGES * tr_stage_words() + tr_common_words());
}

} // namespace wl_tma

// Pools the bulk-copy runner takes: n = 4 and N in [TR_MIN_N, 2^28] (32-bit
// lane, span and slot offsets; a span of alpha T <= N values wraps at most
// once: wl_run_tma caps T at N / max alpha, which binds only below 16384).
// A pass whose strides have lcm above TR_LMAX runs the plain gather instead.
// Other pools take the per-thread runners.  From 4096 on the runner beat the
// per-thread path (pools of 2^8 to 2^14, frac = 1: 0.0738 against 0.0945 ms
// per batched pass; 2048 timed the same).
#ifndef TR_MIN_N
#define TR_MIN_N 4096
#endif
__host__ __device__ inline bool wl_tma_run_eligible(int n, int64_t N)
{
    return n == 4 && N >= TR_MIN_N && N <= ((int64_t)1 << 28);
}

// Lane tables of one pass into `tab` (a tr_common_words() area): J[L + 1]
// lane starts, lanebase[4][TR_LMAX] (slot position of each lane's first
// value, before its span's lead, in bits 8.., its span in bits 0..7) and
// spanC[spans] (span starts).  They depend on N, the strides (their lcm L)
// and the tile length T only.  Every thread of the CTA calls; the caller
// orders the previous readers of `tab` before the call and the new readers
// after it (barriers).
__device__ inline void wl_tma_tables(int64_t N, int L, int T, const int32_t *alpha, int *tab)
{
    using namespace wl_tma;
    const int tid = threadIdx.x;
    int m[4], sb[5], SL[4], slot0[4];
    sb[0] = 0;
    slot0[0] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        m[i] = tm_divc(L, alpha[i]);
        sb[i + 1] = sb[i] + m[i];
        SL[i] = (alpha[i] * T + TR_SPAN_PAD) & ~3;
        if (i < 3)
            slot0[i + 1] = slot0[i] + m[i] * ((alpha[i] * T + TR_SPAN_PAD) & ~3);
    }
    const int nspans = sb[4];
    int *J = tab;
    int *lanebase = J + (TR_LMAX + 1);
    int *spanC = lanebase + 4 * TR_LMAX;
    const int N32 = (int)N;
    for (int l = tid; l <= L; l += blockDim.x) {
        const int qN = tm_divc(N32, L), rN = N32 - qN * L;
        J[l] = l * qN + tm_divc(l * rN + L - 1, L);
    }
    for (int s = tid; s < nspans; s += blockDim.x) {
        const int i = tm_sub<4>(s, sb);
        const int p = s - sb[i], mi = m[i];
        const int qN = tm_divc(N32, mi), rN = N32 - qN * mi;
        spanC[s] = p * qN + tm_divc(p * rN + mi - 1, mi);
    }
    __syncthreads();
    for (int e = tid; e < 4 * L; e += blockDim.x) {
        int i = tm_divc(e, L), l = e - i * L;
        int w = tm_divc(l, m[i]), p = l - w * m[i];
        int64_t r = (int64_t)alpha[i] * J[l] - (int64_t)w * N - spanC[sb[i] + p];
        lanebase[i * TR_LMAX + l] = ((slot0[i] + p * SL[i] + (int)r) << 8) | (sb[i] + p);
    }
    __syncthreads();
}

// Tile length (lane times) of a pass with L lanes: the ring's memory as two
// stages, or as one stage of twice the length from TR_ONE_STAGE_L lanes on
// (see wl_tma_pass_cta), capped at tcap.
__device__ __forceinline__ int wl_tma_tile_T(int L, int tcap)
{
    const int S = L >= TR_ONE_STAGE_L ? 1 : TR_STAGES;
    return min(wl_tma::tm_divc(TR_ETARGET * TR_STAGES / S, L), tcap);
}

// One pass src -> dst of an n = 4 pool (a pool wl_tma_run_eligible accepts)
// whose strides have lcm L <= TR_LMAX.  Every thread of the CTA calls; the
// terms of its values are added to (lo, hi) and its bad-value flag to `bad`.
// The pass's returned values [0, w1) go to o (o may be null when w1 == 0).
//
// Spans: each bulk copy starts at the 16-byte boundary at or below the span's
// first address (its lead, 0..3 values, is recorded per stage).  A span that
// runs past the end of its row is copied in two parts: [as, N4) with N4 = N
// rounded up to a multiple of 4 (the row pitch leaves room past N), then the
// wrapped part from the row start, placed right after it.  Values of the span
// at slot positions from N - as on therefore sit N4 - N further on: each span
// records that threshold and shift, and the consumers add the shift to
// positions at or past the threshold (the shift is 0 when 4 divides N).
//
// tile0, tstep, tcap: this CTA takes tiles tile0, tile0 + tstep, ... of the
// pass (a grid of CTAs sharing one pool), each of at most tcap lane times;
// the defaults take every tile at the ring's full length.  pre: the pass's
// lane tables already built by wl_tma_tables (same L and T), else they are
// built here in the ring's own table area.  SG, signs: the generator draws a
// sign pattern each pass (matrix A D_k; bit i negates g_i); without SG the
// kernel carries no sign code.
template <bool SG = false>
__device__ inline void wl_tma_pass_cta(const float *src, float *dst, int64_t N, int64_t Np, int L,
                                       const int32_t *alpha, const int64_t *gam, float c, float *o,
                                       int64_t w1, float mu, float sigma, float *smem, WlTmaRing &ring,
                                       WlDevState *st, uint64_t &lo, uint64_t &hi, uint32_t &bad,
                                       int tile0 = 0, int tstep = 1, int tcap = 1 << 30,
                                       const int *pre = nullptr, uint32_t signs = 0)
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
    // Large lane counts leave lanes of few values per tile, and their short
    // store runs end in partially written sectors that L2 completes by
    // reading DRAM; there the ring's memory forms one stage of twice the
    // lane times (the consumers, not the copies, set the pace of such pools)
    const int S = L >= TR_ONE_STAGE_L ? 1 : TR_STAGES;
    const int SW = TR_STAGES * tr_stage_words() / S;   // words per stage
    const int SDW = SW - 2 * TR_MAXSPANS;               // span data words per stage
    const int T = wl_tma_tile_T(L, tcap);
    int SL[4], slot0[4];
    slot0[0] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        SL[i] = (alpha[i] * T + TR_SPAN_PAD) & ~3;   // 16-byte aligned slots
        if (i < 3)
            slot0[i + 1] = slot0[i] + m[i] * SL[i];
    }
    float *stage0 = smem;
    int *common = pre ? (int *)pre : (int *)(smem + TR_STAGES * tr_stage_words());
    const int *J = common;
    const int *lanebase = J + (TR_LMAX + 1);
    const int *spanC = lanebase + 4 * TR_LMAX;
    const int N32 = (int)N;
    if (!pre) {
        // the previous pass's readers of the tables are done
        __syncthreads();
        wl_tma_tables(N, L, T, alpha, common);
    }
    const int maxlen = tm_divc(N32 + L - 1, L);
    const int ntiles = (maxlen + T - 1) / T;
    // this CTA's kt-th tile (tile0 + kt tstep) uses stage kt % S for the
    // (uses[s] + kt / S)-th time
    const int nmine = ntiles > tile0 ? (ntiles - tile0 + tstep - 1) / tstep : 0;
    int use[TR_STAGES];
#pragma unroll
    for (int q = 0; q < TR_STAGES; q++)
        use[q] = ring.uses[q];
    const int N4 = (N32 + 3) & ~3;

    if (warp >= TM_CONS_WARPS) {
        // ---------------- producer warps: spans ptid, ptid + 128 (KS per thread) ----------------
        const int ptid = (warp - TM_CONS_WARPS) + TM_PROD_WARPS * lane;
        auto produce = [&](auto ksc) {
            constexpr int KS = decltype(ksc)::value;
            int sp_alpha[KS];
            int64_t sp_gam[KS], sp_C[KS];
            uint32_t sp_doff[KS];
            const float *sp_row[KS];
#pragma unroll
            for (int k = 0; k < KS; k++) {
                const int sp = ptid + 32 * TM_PROD_WARPS * k;
                sp_alpha[k] = 0;
                sp_gam[k] = 0;
                sp_C[k] = 0;
                sp_doff[k] = 0;
                sp_row[k] = src;
                if (sp < nspans) {
                    const int i = tm_sub<4>(sp, sb);
                    const int p = sp - sb[i];
                    sp_alpha[k] = alpha[i];
                    sp_gam[k] = gam[i];
                    sp_C[k] = spanC[sp];
                    sp_doff[k] = (uint32_t)(slot0[i] + p * SL[i]);
                    sp_row[k] = src + (int64_t)i * Np;
                }
            }
            const uint32_t stage_base = smem_u32(stage0);
            // the stage layout may differ from the previous pass's: order the
            // consumers' reads of this memory (before the pass's first
            // barrier) before this pass's bulk copies into it
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            int issued[TR_STAGES];   // uses of each stage this thread issued copies for, + 1
#pragma unroll
            for (int q = 0; q < TR_STAGES; q++)
                issued[q] = 0;
            for (int kt = 0; kt < nmine; kt++) {
                const int tile = tile0 + kt * tstep;
                const int s = S == 1 ? 0 : kt % TR_STAGES;
                int u = use[0];
#pragma unroll
                for (int q = 1; q < TR_STAGES; q++)
                    u = s == q ? use[q] : u;   // (constant indices: no local memory)
                u += S == 1 ? kt : kt / TR_STAGES;
                if (*ring.abort_flag)
                    break;
                if (u > 0 && !mbar_wait(smem_u32(&ring.empty[s]), (uint32_t)((u - 1) & 1))) {
                    *ring.abort_flag = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int t0 = tile * T;
                const int Tt = min(T, maxlen - t0);
                float *sdata = stage0 + s * SW;
                int *info0 = (int *)(sdata + SDW);   // lead | shift << 2
                int *info1 = info0 + TR_MAXSPANS;                       // wrap threshold (slot position)
                const uint32_t full = smem_u32(&ring.full[s]);
                const uint32_t dbase = stage_base + 4u * (uint32_t)(s * SW);
                int as[KS], e2[KS];
                uint32_t b1[KS];
                uint32_t total = 0;
#pragma unroll
                for (int k = 0; k < KS; k++) {
                    const int sp = ptid + 32 * TM_PROD_WARPS * k;
                    as[k] = 0;
                    e2[k] = 0;
                    b1[k] = 0;
                    if (sp < nspans) {
                        int64_t addr = sp_C[k] + (int64_t)sp_alpha[k] * t0 + sp_gam[k];   // < 3N
                        if (addr >= N)
                            addr -= N;
                        if (addr >= N)
                            addr -= N;
                        const int len = sp_alpha[k] * Tt;
                        as[k] = (int)addr & ~3;
                        if (addr + len > N) {
                            // [as, N4), then [0, e2) at slot position N4 - as
                            e2[k] = ((int)(addr + len - N) + 3) & ~3;
                            b1[k] = 4u * (uint32_t)(N4 - as[k]);
                            info0[sp] = ((int)addr - as[k]) | ((N4 - N32) << 2);
                            info1[sp] = (int)sp_doff[k] + (N32 - as[k]);
                        } else {
                            b1[k] = 16u * (uint32_t)(((int)addr - as[k] + len + 3) >> 2);
                            info0[sp] = (int)addr - as[k];
                            info1[sp] = 0x7fffffff;
                        }
                        total += b1[k] + 4u * (uint32_t)e2[k];
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    total += __shfl_xor_sync(0xffffffffu, total, off);
                if (lane == 0)
                    mbar_expect_tx(full, total);
                __syncwarp();
#pragma unroll
                for (int k = 0; k < KS; k++) {
                    if (b1[k]) {
                        const uint32_t d = dbase + 4u * sp_doff[k];
                        bulk_g2s(d, sp_row[k] + as[k], b1[k], full);
                        if (e2[k])
                            bulk_g2s(d + b1[k], sp_row[k], 4u * (uint32_t)e2[k], full);
                    }
                }
                mbar_arrive(full);
#pragma unroll
                for (int q = 0; q < TR_STAGES; q++)
                    if (s == q)
                        issued[q] = u + 1;
            }
            if (*ring.abort_flag) {
                // copies still in flight must land before the CTA moves on
#pragma unroll
                for (int q = 0; q < TR_STAGES; q++)
                    if (issued[q] > 0 && !mbar_wait(smem_u32(&ring.full[q]), (uint32_t)((issued[q] - 1) & 1)))
                        atomicOr(&st->status, WL_ETIMEOUT);
            }
        };
        if (nspans > 32 * TM_PROD_WARPS)
            produce(std::integral_constant<int, 2>{});
        else
            produce(std::integral_constant<int, 1>{});
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
        // transform, store, sum of squares and returned values of one tuple
        auto emit = [&](const float *gv, int64_t j, uint64_t &tl, uint32_t &emax) {
            float y[4];
            wl_xform4(gv, c, y);
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
                dstk[kk][j] = y[kk];
                tl += term32(y[kk], emax);
                if (ret[kk]) {
                    outk[kk][j] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                } else {
                    const int64_t q = kk * N + j;
                    if (q < w1)
                        o[q] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                }
            }
        };
        const uint32_t magicT = tl_magic((uint32_t)T);
        uint32_t emax = 0;
        const bool shifted = N4 != N32;   // wrapped spans sit shifted past their threshold
        {
            for (int kt = 0; kt < nmine; kt++) {
                const int tile = tile0 + kt * tstep;
                const int s = S == 1 ? 0 : kt % TR_STAGES;
                int u = use[0];
#pragma unroll
                for (int q = 1; q < TR_STAGES; q++)
                    u = s == q ? use[q] : u;
                u += S == 1 ? kt : kt / TR_STAGES;
                if (*ring.abort_flag)
                    break;
                if (!mbar_wait(smem_u32(&ring.full[s]), (uint32_t)(u & 1))) {
                    *ring.abort_flag = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int t0 = tile * T;
                const int Tt = min(T, maxlen - t0);
                const float *sdata = stage0 + s * SW;
                const int *info0 = (const int *)(sdata + SDW);
                const int *info1 = info0 + TR_MAXSPANS;
                uint64_t tl = 0;   // this tile's terms: a few hundred per thread at most, each below 2^48
                // long lanes: each warp owns whole lanes, 64 lane times per
                // step; lane l of tile k goes to warp (k L + l) mod 15, so when
                // 15 does not divide L the extra lanes rotate over the warps
                auto lane_loop = [&](auto shc, auto sgc) {
                    constexpr bool SH = decltype(shc)::value;
                    constexpr bool SG = decltype(sgc)::value;
                    int l0 = warp - (int)(((uint32_t)tile * (uint32_t)L) % TM_CONS_WARPS);
                    l0 += l0 < 0 ? TM_CONS_WARPS : 0;
                    for (int l = l0; l < L; l += TM_CONS_WARPS) {
                        const int jl = J[l];
                        const int tmax = min(Tt, J[l + 1] - jl - t0);
                        int gb[4], thr[4], sh[4];
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            const int lb = lanebase[i * TR_LMAX + l];
                            const int f0 = info0[lb & 255];
                            gb[i] = (lb >> 8) + (f0 & 3);
                            sh[i] = f0 >> 2;
                            thr[i] = info1[lb & 255];
                        }
                        const int64_t jb = (int64_t)jl + t0;
                        for (int t = lane; t < tmax; t += 64) {
                            // two independent values per thread: t and t + 32
                            const bool v2 = t + 32 < tmax;
                            float gv[4], hv[4];
#pragma unroll
                            for (int i = 0; i < 4; i++) {
                                int q = gb[i] + alpha[i] * t;
                                int q2 = q + alpha[i] * 32;
                                if constexpr (SH) {
                                    q += q >= thr[i] ? sh[i] : 0;
                                    q2 += q2 >= thr[i] ? sh[i] : 0;
                                }
                                gv[i] = sdata[q];
                                hv[i] = v2 ? sdata[q2] : 0.f;
                                if (SG) {   // the pass's matrix is A D_k
                                    gv[i] = wl_sgn(gv[i], signs, i);
                                    hv[i] = wl_sgn(hv[i], signs, i);
                                }
                            }
                            // both tuples' stores interleaved: each row gets
                            // 256 contiguous bytes per warp at once
                            float y[4], z[4];
                            wl_xform4(gv, c, y);
                            wl_xform4(hv, c, z);
                            const int64_t j = jb + t;
#pragma unroll
                            for (int kk = 0; kk < 4; kk++) {
                                dstk[kk][j] = y[kk];
                                if (v2)
                                    dstk[kk][j + 32] = z[kk];
                                tl += term32(y[kk], emax);
                                if (v2)
                                    tl += term32(z[kk], emax);
                                if (ret[kk]) {
                                    outk[kk][j] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                                    if (v2)
                                        outk[kk][j + 32] = __fadd_rn(mu, __fmul_rn(sigma, z[kk]));
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
                };
                if (T >= TR_LANE_MIN_T) {
                    if (shifted)
                        lane_loop(std::true_type{}, std::integral_constant<bool, SG>{});
                    else
                        lane_loop(std::false_type{}, std::integral_constant<bool, SG>{});
                } else {
                    // short tiles: threads take (lane, time) pairs, times fastest
                    const int npairs = L * T;
                    for (int f = tid; f < npairs; f += TM_CONS_THREADS) {
                        const int l = (int)tl_div((uint32_t)f, (uint32_t)T, magicT);
                        const int t = f - l * T;
                        const int jl = J[l];
                        if (t >= Tt || t0 + t >= J[l + 1] - jl)
                            continue;
                        float gv[4];
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            const int lb = lanebase[i * TR_LMAX + l];
                            const int f0 = info0[lb & 255];
                            int q = (lb >> 8) + (f0 & 3) + alpha[i] * t;
                            q += q >= info1[lb & 255] ? (f0 >> 2) : 0;
                            gv[i] = SG ? wl_sgn(sdata[q], signs, i) : sdata[q];
                        }
                        emit(gv, (int64_t)jl + t0 + t, tl, emax);
                    }
                }
                lo += tl;
                hi += lo < tl ? 1ull : 0ull;
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(smem_u32(&ring.empty[s]));
            }
        }
        bad |= emax >= 135u ? 1u : 0u;
        // the next pass reads this pool with bulk copies (the async proxy)
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
    }
    // the uses every thread counted, the same in all of them
    // stage q served the tiles kt = q, q + S, ... of this pass
#pragma unroll
    for (int q = 0; q < TR_STAGES; q++)
        ring.uses[q] = use[q] + (q < S ? (nmine + S - 1 - q) / S : 0);
}

// out[q] = mu + sigma pool[q] for q < w1 (logical positions; rows of N at
// pitch Np): the returned values of the pass that just wrote `pool`, read
// back while it is still in L2.  Consecutive threads take consecutive
// values, eight loads in flight per thread.  Every thread of the CTA calls,
// after a barrier that follows the pass's stores.
static __device__ __noinline__ void wl_return_copy(const float *pool, int64_t N, int64_t Np, int64_t w1, float *o, float mu,
                                      float sigma)
{
    const int B = blockDim.x;
    for (int k = 0; k < 4 && (int64_t)k * N < w1; k++) {
        const int n = (int)min(N, w1 - (int64_t)k * N);
        const float *row = pool + k * Np;
        float *ok = o + (int64_t)k * N;
        int j = threadIdx.x;
        for (; j + 7 * B < n; j += 8 * B) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; u++)
                v[u] = __ldcg(row + j + u * B);
#pragma unroll
            for (int u = 0; u < 8; u++)
                ok[j + u * B] = __fadd_rn(mu, __fmul_rn(sigma, v[u]));
        }
        for (; j < n; j += B)
            ok[j] = __fadd_rn(mu, __fmul_rn(sigma, __ldcg(row + j)));
    }
}

// All passes of the spec (a pool wl_tma_run_eligible accepts) from global
// memory through the bulk-copy pass; a pass whose strides have lcm above
// TR_LMAX takes the plain gather.  Returns the index of the buffer holding the
// final pool.
template <bool SG = false>
__device__ inline int wl_run_tma(const WlRunSpec &d, float *smem, uint64_t *red,
                                 WlTmaRing &ring)
{
    const int tid = threadIdx.x;
    const int64_t N = d.N, nu = 4 * N;
    const double rnu = wl_rnu(nu);
    int cur = d.cur;
    WlDevState *st = d.st;   // the CTA's shared-memory copy of the state
    for (int64_t p = 0; p < d.passes; p++) {
        // parameters as the previous pass's end (a barrier) left them
        if (tid == 0)
            st->last = st->next;
        int32_t alpha[4];
        int64_t gam[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
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
        const int L = wl_lcm4(alpha);
        const bool tma = L <= TR_LMAX && !*ring.abort_flag;
        // a span of a tile holds alpha T values: at most N, so it wraps at most once
        const int amax = max(max(alpha[0], alpha[1]), max(alpha[2], alpha[3]));
        const int tcap = max(1, (int)(N / amax));
        // the plain gather below writes its returned values itself
        const bool copy_back = tma && L >= TR_RETURN_COPY_L && o && w1 > 0;
        if (tma) {
            wl_tma_pass_cta<SG>(src, dst, N, d.Np, L, alpha, gam, c, copy_back ? nullptr : o, copy_back ? 0 : w1,
                                d.mu, d.sigma, smem, ring, d.st, lo, hi, bad, 0, 1, tcap, nullptr,
                                st->next.signs);
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
            job.signs = SG ? st->next.signs : 0u;
            job.out = o;
            job.w0 = 0;
            job.w1 = w1;
            job.mu = d.mu;
            job.sigma = d.sigma;
            wl_gather4_range(job, tid, blockDim.x, lo, hi, bad);
            // the next pass may read this pool with bulk copies
            asm volatile("fence.proxy.async.global;\n" ::: "memory");
        }
        const float *xp = &dst[wl_last_phys(4, N, d.Np)];
        wl_end_pass_cta(st, 4, N, nu, rnu, lo, hi, bad, red, [xp]() { return (double)__ldcg(xp); }, st->msigns,
                        false);
        if (copy_back)
            wl_return_copy(dst, N, d.Np, w1, o, d.mu, d.sigma);
        cur = 1 - cur;
    }
    return cur;
}
