// One pass of Wallace's generator for n = 8 (A = J/4 - I in Eq. 1 of Brent's
// RANN4 paper), binary32 pool, N a multiple of 4 and coprime to 105, as a
// warp-specialised lane-tiled gather fed by bulk (TMA) copies: the n = 8
// member of the family in wl_tiled_tma.cu.
//
// Geometry.  With N coprime to 105 a pass draws eight distinct strides from
// the eleven odd divisors of 315 = 3^2 5 7 above one.  Any eight of them
// include a multiple of 9, one of 5 and one of 7, so every pass has
// L = lcm(alpha_i) = 315 lanes.  Lane l covers j in [J_l, J_l+1),
// J_l = ceil(l N / L); a tile of T = 8 lane times reads, per sub-vector i,
// m_i = L / alpha_i contiguous spans of 8 alpha_i values (span p starts at
// ceil(p N / m_i) + alpha_i t0 + gamma_i mod N) and uses every value it
// reads: at most 105 + 63 + 45 + 35 + 21 + 15 + 9 + 7 = 300 spans of 96 B to
// 10 KB.  A tile is 8 x 315 x 8 values (80 KB); two stages of it and their
// slack take 180 KB of shared memory, which is what holds T at 8.  A lane's
// store run per tile is therefore 32 bytes and mostly half sectors (the
// neighbouring tile, taken by another CTA at about the same time, writes the
// rest of each sector while it is still in L2); these stores set the pace.
// For pools over 64 MB the returned values are not stored beside the pool but
// copied from the new pool after the pass by a streaming kernel
// (t8_return_kernel, float4 where the output allows).
//
// Pipeline as in the n = 4 kernel: one persistent CTA per SM, tiles handed
// out from the generator's counter; producer threads each own up to T8_KS
// spans for the whole pass and issue one bulk copy per span (two where it
// wraps past the end of its row); consumer warps take items of 4 lanes x 8
// lane times (one value of every sub-vector per thread, so a store
// instruction writes four 32-byte runs), dealt round-robin over the warps and
// rotated from tile to tile.  Every wait is bounded; on expiry the CTA
// records WALLACE_ETIMEOUT, stops issuing work, waits (bounded) for its own
// copies still in flight, and leaves.
#include <math.h>

#include "wl_common.cuh"
#include "wl_launch.h"
#include "wl_tma_common.cuh"

#define T8_L 315                  /* lanes: lcm of any eight divisors of 315 above one */
#define T8_T 8                    /* lane times per tile */
#define T8_STAGES 2
#define T8_MAXSPANS 300           /* sum of 315 / alpha over the eight smallest candidates */
#define T8_SPAN_PAD 8             /* slot words past 8 alpha: alignment lead and a wrap's rounding */
#define T8_CONS_WARPS 20          /* 15 and 24 time 3% slower */
#define T8_PROD_WARPS 4           /* 8 warps time the same */
#define T8_KS ((T8_MAXSPANS + 32 * T8_PROD_WARPS - 1) / (32 * T8_PROD_WARPS))
#define T8_THREADS (32 * (T8_CONS_WARPS + T8_PROD_WARPS))
#define T8_GROUPS ((T8_L + 3) / 4)   /* consumer items per tile, 4 lanes each */
// a stage: the span slots (sum_i m_i (8 alpha_i + 8) <= 8 * 315 * 8 + 8 * 300
// words), then every span's alignment lead; rounded up to 128 bytes
#define T8_SDW (8 * T8_L * T8_T + T8_SPAN_PAD * T8_MAXSPANS)
#define T8_SW (((T8_SDW + T8_MAXSPANS) + 31) & ~31)
// common area: J[L + 1], lane table [8][L], per span its start, slot and sub-vector
#define T8_CW ((T8_L + 1) + 8 * T8_L + 3 * T8_MAXSPANS)
#define T8_SMEM_BYTES (4 * (T8_STAGES * T8_SW + T8_CW))
// pools above this size leave the returned values to a streaming kernel
// after the pass; smaller ones stay in L2, where the half-sector stores of
// a lane's 8-value runs merge cheaply
#ifndef T8_RETURN_KERNEL_BYTES
#define T8_RETURN_KERNEL_BYTES (64ll << 20)
#endif

static_assert(T8_SMEM_BYTES <= 227 * 1024 - 2048, "stage ring exceeds shared memory");
static_assert((T8_SW * 4) % 128 == 0, "stages must stay 128-byte aligned");
static_assert(32 * T8_PROD_WARPS * T8_KS >= T8_MAXSPANS, "producer threads cannot hold every span");
static_assert(T8_STAGES == 2, "the producers track two stages");

namespace {

using namespace wl_tma;

// Wait for the previous pass (its pool, state and scale visible), let the
// next pass's CTAs launch, and return this pass's scale c.
__device__ __forceinline__ float t8_wait_prev(WlDevState *st, volatile float *s_c)
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    if (threadIdx.x == 0)
        *s_c = __ldcg(&st->next.c32);
    __syncthreads();
    return *s_c;
}

// SG: the generator draws a sign pattern each pass (matrix A D_k).
template <bool SG>
__global__ void __launch_bounds__(T8_THREADS, 1) tma8_kernel(WlPassArgs a, double rnu)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar_full[T8_STAGES];
    __shared__ __align__(8) uint64_t bar_empty[T8_STAGES];
    __shared__ __align__(8) uint64_t bar_tile[T8_STAGES];   // a stage's tile index is published
    __shared__ volatile int s_stage_tile[T8_STAGES];
    __shared__ uint64_t red[3 * (T8_THREADS / 32 + 1)];
    __shared__ volatile int s_abort;
    __shared__ int64_t s_gam[8];
    __shared__ int s_alpha[8];
    __shared__ uint32_t s_signs;
    __shared__ volatile float s_c;

    // Launched as a programmatic dependent of the previous pass: everything
    // up to t8_wait_prev() uses only this pass's strides, drawn two
    // finalisers back; the pool and the scale c are read after the wait.
    WlDevState *st = a.st;
    const float *__restrict__ src = (const float *)a.src;
    float *__restrict__ dst = (float *)a.dst;
    const int64_t N = a.N, Np = a.Np;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        const WlStrides *cur = &st->ahead[a.pass & 1];
        if (lane < 8)
            s_alpha[lane] = __ldcg(&cur->alpha[lane]);
        else if (lane < 16)
            s_gam[lane - 8] = (int64_t)__ldcg((const long long *)&cur->gamma[lane - 8]);
        else if (lane == 16)
            s_signs = SG ? __ldcg(&cur->signs) : 0u;
    }
    __syncthreads();
    const uint32_t signs = SG ? s_signs : 0u;
    int alpha[8];
#pragma unroll
    for (int i = 0; i < 8; i++)
        alpha[i] = s_alpha[i];

    // every stride divides 315 when N is coprime to 105; any other set (not
    // drawn for such N) takes the plain gather below
    bool tileable = true;
    int e3 = 0, e5 = 0, e7 = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int al = alpha[i];
        tileable &= al > 1 && al <= T8_L && T8_L % al == 0;
        e3 = max(e3, al % 9 == 0 ? 2 : (al % 3 == 0 ? 1 : 0));
        e5 |= al % 5 == 0 ? 1 : 0;
        e7 |= al % 7 == 0 ? 1 : 0;
    }
    tileable &= e3 == 2 && e5 == 1 && e7 == 1;
    int m[8], sb[9];
    sb[0] = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        m[i] = tileable ? T8_L / alpha[i] : 0;
        sb[i + 1] = sb[i] + m[i];
    }
    const int nspans = sb[8];

    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    float *out = (float *)a.out;
    const float mu = (float)a.mu, sigma = (float)a.sigma;
    const int64_t w0 = a.w0, w1 = a.w1;
    float c;

    if (!tileable || nspans > T8_MAXSPANS || N < TM_MIN_N || (N & 3)) {
        // plain strided gather for this pass
        c = t8_wait_prev(st, &s_c);
        const int64_t G = (int64_t)gridDim.x * blockDim.x;
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + tid; j < N; j += G) {
            float g[8], y[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int64_t ix = (int64_t)(((uint64_t)alpha[i] * (uint64_t)j + (uint64_t)s_gam[i]) % (uint64_t)N);
                g[i] = SG ? wl_sgn(src[i * Np + ix], signs, i) : src[i * Np + ix];
            }
            wl_xform8(g, c, y);
#pragma unroll
            for (int k = 0; k < 8; k++) {
                dst[k * Np + j] = y[k];
                wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                const int64_t q = k * N + j;
                if (q >= w0 && q < w1)
                    out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, y[k]));
            }
        }
    } else {
        float *stage0 = smem;
        int *common = (int *)(smem + T8_STAGES * T8_SW);
        int *J = common;                          // [L + 1] lane starts
        int *lanetab = J + (T8_L + 1);            // [8][L]: slot word of the lane's first value << 9 | span
        int *spanC = lanetab + 8 * T8_L;          // [spans]: ceil(p N / m_i)
        int *spanOff = spanC + T8_MAXSPANS;       // [spans]: slot offset in a stage, words
        int *spanSub = spanOff + T8_MAXSPANS;     // [spans]: sub-vector
        int slot0[8];
        slot0[0] = 0;
#pragma unroll
        for (int i = 0; i < 7; i++)
            slot0[i + 1] = slot0[i] + m[i] * (T8_T * alpha[i] + T8_SPAN_PAD);

        // ceil(l N / L) as l (N / L) + ceil(l (N mod L) / L): 32-bit
        // arithmetic (N <= 2^28, l (N mod L) < L^2)
        const int N32 = (int)N;
        {
            const int qL = N32 / T8_L, rL = N32 - qL * T8_L;
            for (int l = tid; l <= T8_L; l += T8_THREADS)
                J[l] = l * qL + (l * rL + T8_L - 1) / T8_L;
        }
        for (int sp = tid; sp < nspans; sp += T8_THREADS) {
            int i = 0, p = 0, mi = 1, al = 1, so = 0;
#pragma unroll
            for (int k = 0; k < 8; k++)
                if (sp >= sb[k] && sp < sb[k + 1]) {
                    i = k;
                    p = sp - sb[k];
                    mi = m[k];
                    al = alpha[k];
                    so = slot0[k];
                }
            const int qN = N32 / mi, rN = N32 - qN * mi;
            spanC[sp] = p * qN + (p * rN + mi - 1) / mi;
            spanOff[sp] = so + p * (T8_T * al + T8_SPAN_PAD);
            spanSub[sp] = i;
        }
        if (tid == 0) {
            for (int s = 0; s < T8_STAGES; s++) {
                mbar_init(smem_u32(&bar_full[s]), 32 * T8_PROD_WARPS);
                mbar_init(smem_u32(&bar_empty[s]), T8_CONS_WARPS);
                mbar_init(smem_u32(&bar_tile[s]), 1);
            }
            s_abort = 0;
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
        __syncthreads();
        // lane l of sub-vector i reads span p = l mod m_i from offset
        // r = alpha_i J_l - floor(l / m_i) N - spanC in [0, alpha_i)
        for (int e = tid; e < 8 * T8_L; e += T8_THREADS) {
            const int i = e / T8_L, l = e - i * T8_L;
            int mi = 1, al = 1, s0 = 0;
#pragma unroll
            for (int k = 0; k < 8; k++)
                if (k == i) {
                    mi = m[k];
                    al = alpha[k];
                    s0 = sb[k];
                }
            const int w = l / mi, p = l - w * mi;
            const int sp = s0 + p;
            const int64_t r = (int64_t)al * J[l] - (int64_t)w * N - spanC[sp];
            lanetab[e] = ((spanOff[sp] + (int)r) << 9) | sp;
        }
        __syncthreads();
        c = t8_wait_prev(st, &s_c);
        const int maxlen = (N32 + T8_L - 1) / T8_L;
        const int ntiles = (maxlen + T8_T - 1) / T8_T;

        if (warp >= T8_CONS_WARPS) {
            // ---------------- producer warps ----------------
            const int pw = warp - T8_CONS_WARPS;
            const int pt = pw + T8_PROD_WARPS * lane;   // spans pt + 32 PW q, q < KS
            const uint32_t stage_base = smem_u32(stage0);
            int issued0 = 0, issued1 = 0;   // per stage: uses issued (phase parity of the last)
            for (int it = 0;; it++) {
                const int s = it & 1, k = it >> 1;
                if (s_abort)
                    break;
                if (k > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (uint32_t)((k - 1) & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                // producer warp 0 takes the next tile from the generator's
                // counter and publishes it
                if (pw == 0) {
                    if (lane == 0) {
                        s_stage_tile[s] = (int)atomicAdd(&st->tile_ctr, 1u);
                        mbar_arrive(smem_u32(&bar_tile[s]));
                    }
                    __syncwarp();
                } else if (!mbar_wait(smem_u32(&bar_tile[s]), (uint32_t)(k & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int tile = s_stage_tile[s];
                const uint32_t full = smem_u32(&bar_full[s]);
                if (tile >= ntiles) {
                    // no more tiles: release the consumers without data
                    mbar_arrive(full);
                    (s ? issued1 : issued0) = k + 1;
                    break;
                }
                const int t0 = tile * T8_T;
                const int Tt = min(T8_T, maxlen - t0);
                int *lead = (int *)(stage0 + s * T8_SW + T8_SDW);
                const uint32_t sbase = stage_base + 4u * (uint32_t)(s * T8_SW);
                int sa[T8_KS], sl[T8_KS], sub[T8_KS], soff[T8_KS];
                uint32_t total = 0;
#pragma unroll
                for (int q = 0; q < T8_KS; q++) {
                    const int sp = pt + 32 * T8_PROD_WARPS * q;
                    sl[q] = 0;
                    sa[q] = 0;
                    sub[q] = 0;
                    soff[q] = 0;
                    if (sp < nspans) {
                        const int i = spanSub[sp];
                        const int al = s_alpha[i];
                        int64_t ad = (int64_t)spanC[sp] + (int64_t)al * t0 + s_gam[i];   // < 3N
                        if (ad >= N)
                            ad -= N;
                        if (ad >= N)
                            ad -= N;
                        sa[q] = (int)ad;
                        sl[q] = al * Tt;
                        sub[q] = i;
                        soff[q] = spanOff[sp];
                        const int as = sa[q] & ~3;
                        lead[sp] = sa[q] - as;
                        total += sa[q] + sl[q] > N32
                                     ? 4u * (uint32_t)(N32 - as) + 4u * (uint32_t)((sa[q] + sl[q] - N32 + 3) & ~3)
                                     : 16u * (uint32_t)((sa[q] - as + sl[q] + 3) >> 2);
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    total += __shfl_xor_sync(0xffffffffu, total, off);
                if (lane == 0)
                    mbar_expect_tx(full, total);
                __syncwarp();
#pragma unroll
                for (int q = 0; q < T8_KS; q++) {
                    if (sl[q] == 0)
                        continue;
                    const float *row = src + (int64_t)sub[q] * Np;
                    const uint32_t d = sbase + 4u * (uint32_t)soff[q];
                    const int as = sa[q] & ~3;
                    if (sa[q] + sl[q] <= N32) {
                        bulk_g2s(d, row + as, 16u * (uint32_t)((sa[q] - as + sl[q] + 3) >> 2), full);
                    } else {
                        bulk_g2s(d, row + as, 4u * (uint32_t)(N32 - as), full);
                        bulk_g2s(d + 4u * (uint32_t)(N32 - as), row,
                                 4u * (uint32_t)((sa[q] + sl[q] - N32 + 3) & ~3), full);
                    }
                }
                mbar_arrive(full);
                (s ? issued1 : issued0) = k + 1;
            }
            // copies still in flight must land before the CTA leaves
            if (issued0 > 0 && !mbar_wait(smem_u32(&bar_full[0]), (uint32_t)((issued0 - 1) & 1)))
                atomicOr(&st->status, WL_ETIMEOUT);
            if (issued1 > 0 && !mbar_wait(smem_u32(&bar_full[1]), (uint32_t)((issued1 - 1) & 1)))
                atomicOr(&st->status, WL_ETIMEOUT);
        } else {
            // ---------------- consumer warps ----------------
            // sub-vectors returned whole, and those returned in part
            uint32_t all_ret = 0, part_ret = 0;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int64_t q0 = k * N, q1 = q0 + N;
                if (q1 > w0 && q0 < w1) {
                    if (q0 >= w0 && q1 <= w1)
                        all_ret |= 1u << k;
                    else
                        part_ret |= 1u << k;
                }
            }
            const int ll = lane >> 3, tt = lane & 7;   // lane of the item, lane time
            uint32_t emax = 0;
            for (int it = 0;; it++) {
                const int s = it & 1, k = it >> 1;
                if (s_abort)
                    break;
                if (!mbar_wait(smem_u32(&bar_full[s]), (uint32_t)(k & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int tile = s_stage_tile[s];
                if (tile >= ntiles)
                    break;
                const int t0 = tile * T8_T;
                const int Tt = min(T8_T, maxlen - t0);
                const float *sdata = stage0 + s * T8_SW;
                const int *lead = (const int *)(sdata + T8_SDW);
                uint64_t tl = 0;   // at most 6 items x 8 terms per thread, each below 2^48
                // item g of tile k goes to warp (k groups + g) mod T8_CONS_WARPS
                int g = warp - (int)(((uint32_t)tile * (uint32_t)T8_GROUPS) % T8_CONS_WARPS);
                g += g < 0 ? T8_CONS_WARPS : 0;
                for (; g < T8_GROUPS; g += T8_CONS_WARPS) {
                    const int l = 4 * g + ll;
                    if (l >= T8_L)
                        continue;
                    const int jl = J[l];
                    if (tt >= min(Tt, J[l + 1] - jl - t0))
                        continue;
                    float x[8], y[8];
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int lb = lanetab[i * T8_L + l];
                        x[i] = sdata[(lb >> 9) + lead[lb & 511] + alpha[i] * tt];
                        if (SG)   // the pass's matrix is A D_k
                            x[i] = wl_sgn(x[i], signs, i);
                    }
                    wl_xform8(x, c, y);
                    const int64_t j = (int64_t)jl + t0 + tt;
#pragma unroll
                    for (int kk = 0; kk < 8; kk++) {
                        dst[kk * Np + j] = y[kk];
                        tl += term32(y[kk], emax);
                        const int64_t q = kk * N + j;
                        if ((all_ret >> kk) & 1u)
                            out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                        else if (((part_ret >> kk) & 1u) && q >= w0 && q < w1)
                            out[q - w0] = __fadd_rn(mu, __fmul_rn(sigma, y[kk]));
                    }
                }
                // a CTA may take any number of tiles: carry into 128 bits
                lo += tl;
                hi += lo < tl ? 1ull : 0ull;
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(smem_u32(&bar_empty[s]));
            }
            bad = emax >= 135u ? 1u : 0u;
        }
    }

    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st))
        wl_finalise_cta(st, 8, N, a.nu, rnu, &dst[wl_last_phys(8, N, Np)], SG ? 1 : 0);
}

// out[q - w0] = mu + sigma pool[q] for the returned window [w0, w1) of the
// new pool (Section 5's returned fraction), row by row; 16-byte accesses where
// the row and the output share their alignment.  Launched as a programmatic
// dependent of the pass: it waits for the pass, then lets the next pass's
// CTAs start their prologue.
__global__ void __launch_bounds__(256) t8_return_kernel(const float *__restrict__ pool, int64_t N, int64_t Np,
                                                        int n, int64_t w0, int64_t w1, float *__restrict__ out,
                                                        float mu, float sigma)
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int k = 0; k < n; k++) {
        const int64_t q0 = max(w0, k * N), q1 = min(w1, k * N + N);
        if (q0 >= q1)
            continue;
        const float *row = pool + k * Np;   // row[q - k N]
        float *o = out + (k * N - w0);      // o[q - k N]
        const int64_t j0 = q0 - k * N, j1 = q1 - k * N;
        if (((uintptr_t)(o + j0) & 15) == ((uintptr_t)(row + j0) & 15)) {
            // scalar head up to the row's 16-byte boundary, then float4
            const int64_t ja = min(j1, (j0 + 3) & ~(int64_t)3);
            const int64_t nv = (j1 - ja) >> 2;
            if (t < ja - j0)
                o[j0 + t] = __fadd_rn(mu, __fmul_rn(sigma, row[j0 + t]));
            const float4 *r4 = (const float4 *)(row + ja);
            float4 *o4 = (float4 *)(o + ja);
            for (int64_t v = t; v < nv; v += G) {
                const float4 y = __ldcs(r4 + v);
                float4 r;
                r.x = __fadd_rn(mu, __fmul_rn(sigma, y.x));
                r.y = __fadd_rn(mu, __fmul_rn(sigma, y.y));
                r.z = __fadd_rn(mu, __fmul_rn(sigma, y.z));
                r.w = __fadd_rn(mu, __fmul_rn(sigma, y.w));
                __stcs(o4 + v, r);
            }
            const int64_t jt = ja + 4 * nv;
            if (t < j1 - jt)
                o[jt + t] = __fadd_rn(mu, __fmul_rn(sigma, row[jt + t]));
        } else {
            for (int64_t j = j0 + t; j < j1; j += G)
                o[j] = __fadd_rn(mu, __fmul_rn(sigma, row[j]));
        }
    }
}

bool g_tma8_configured[2] = {false, false};

} // namespace

bool wl_tma8_supported(int n, int64_t N, int fp64)
{
    // strides divide 315 (N coprime to 105); lane starts, span starts and
    // slot offsets are held in 32-bit integers
    return n == 8 && !fp64 && N >= TM_MIN_N && (N & 3) == 0 && N % 3 != 0 && N % 5 != 0 &&
           N % 7 != 0 && N <= ((int64_t)1 << 28);
}

bool wl_tma8_return_kernel(const WlPassArgs &a)
{
    return a.w1 > a.w0 && (int64_t)sizeof(float) * a.n * a.N > T8_RETURN_KERNEL_BYTES;
}

cudaError_t wl_launch_tma8(const WlPassArgs &a, int sm_count, int signs, cudaStream_t stream)
{
    const int which = signs ? 1 : 0;
    auto kern = which ? tma8_kernel<true> : tma8_kernel<false>;
    if (!g_tma8_configured[which]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T8_SMEM_BYTES);
        if (e != cudaSuccess)
            return e;
        g_tma8_configured[which] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sm_count);
    cfg.blockDim = dim3(T8_THREADS);
    cfg.dynamicSmemBytes = T8_SMEM_BYTES;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const double rnu = sqrt(2.0 * (double)a.nu - 1.0);   // IEEE square root: correctly rounded
    // large pools: the pass writes the new pool only, and the returned values
    // follow in a streaming kernel (in the pass they would be a lane's 8-value
    // runs: half-sector stores)
    const bool split = wl_tma8_return_kernel(a);
    WlPassArgs p = a;
    if (split)
        p.w0 = p.w1 = 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, p, rnu);
    if (e != cudaSuccess || !split)
        return e != cudaSuccess ? e : cudaGetLastError();
    return wl_launch_t8_return(a, sm_count, stream);
}

cudaError_t wl_launch_t8_return(const WlPassArgs &a, int sm_count, cudaStream_t stream)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t rc = {};
    rc.gridDim = dim3(4 * sm_count);
    rc.blockDim = dim3(256);
    rc.stream = stream;
    rc.attrs = attr;
    rc.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&rc, t8_return_kernel, (const float *)a.dst, a.N, a.Np, a.n, a.w0, a.w1,
                                       (float *)a.out, (float)a.mu, (float)a.sigma);
    if (e != cudaSuccess)
        return e;
    return cudaGetLastError();
}
