// One pass of Wallace's generator for n = 8 (A = J/4 - I in Eq. 1 of Brent's
// RANN4 paper), binary32 pool, N a multiple of 4 and coprime to 105, on
// clusters of two CTAs: CTA rank r holds sub-vectors 4r .. 4r + 3 of every
// tile, so a tile can be 315 lanes by T = 16 lane times (each CTA's half of
// it is the size of the one-CTA kernel's whole 8-lane-time tile).  A lane's
// store run per tile is then 64 bytes (three sectors for two of data) where
// the one-CTA kernel (wl_tiled_tma8.cu) writes 32-byte, half-sector runs, and
// each CTA gathers, transforms and sums the squares of four values per tuple.
//
// Geometry as in wl_tiled_tma8.cu: L = 315 lanes, lane l covers j in
// [J_l, J_{l+1}), J_l = ceil(l N / L); for sub-vector i the tile reads
// m_i = L / alpha_i contiguous spans of 16 alpha_i values.
//
// The transform needs every tuple's full sum: with g the pass's gathered
// values (sign-flipped for A D_k), ab = (g0 + g1) + (g2 + g3) on rank 0 and
// de = (g4 + g5) + (g6 + g7) on rank 1, h = (ab + de) / 4 and
// y_k = (h - g_k) c -- the operations of the one-CTA kernel, in its order
// (binary32 addition commutes, so either CTA may add the two halves).  Each
// CTA computes its half-sum for every tuple of the tile (phase 1), stores it
// into its partner's shared memory (a distributed shared memory store), and
// after the partner's half-sums have arrived computes h and its four outputs
// (phase 2).  The exchange is per warp: consumer warp w of both CTAs takes
// the same items of every tile, keeps its four values per tuple in registers
// (so it frees the stage right after phase 1, before any store), and waits
// only for warp w of the partner.  Each warp has two exchange slots, used by
// alternate tiles, in the partner's shared memory, and per slot an mbarrier
// in its own that the partner warp's 32 threads arrive at (remotely, release
// at cluster scope) once they have stored that tile's half-sums; the wait on
// it acquires at cluster scope.  (One barrier for both slots could complete
// the next tile's phase before its waiter looked at this one, and a parity
// wait would then miss it.)  A warp writes slot k mod 2 for tile k only after
// it has received the partner warp's half-sums of tile k - 1, which the
// partner stored after reading slot (k - 2) mod 2 = k mod 2: two slots need
// no second barrier.
//
// Tiles are assigned statically (cluster c takes tiles c, c + C, ...) so the
// two CTAs of a cluster need no shared counter.  The sum of squares goes to
// the generator's accumulators from both CTAs and the last CTA of the grid
// (by ticket) runs the end of pass, as in the other pass kernels.  Every wait
// on an mbarrier is bounded (about a second): on expiry the CTA records
// WALLACE_ETIMEOUT, stops, waits (bounded) for its own bulk copies in flight,
// and reaches the final cluster barrier, which every path reaches, so
// neither CTA leaves while its partner may still write to its shared memory.
#include <math.h>

#include "wl_common.cuh"
#include "wl_launch.h"
#include "wl_tma_common.cuh"

#define C8_L 315                 /* lanes: lcm of any eight divisors of 315 above one */
#define C8_T 16                  /* lane times per tile */
#define C8_STAGES 2
#define C8_MAXSPANS 248          /* a CTA's four sub-vectors: at most 105 + 63 + 45 + 35 spans */
#define C8_SPAN_PAD 8            /* slot words past 16 alpha: alignment lead and a wrap's rounding */
#define C8_CONS_WARPS 20
#define C8_PROD_WARPS 4
#define C8_KS ((C8_MAXSPANS + 32 * C8_PROD_WARPS - 1) / (32 * C8_PROD_WARPS))
#define C8_THREADS (32 * (C8_CONS_WARPS + C8_PROD_WARPS))
#define C8_GROUPS ((C8_L + 1) / 2)   /* consumer items per tile: 2 lanes x 16 lane times */
#define C8_IPW ((C8_GROUPS + C8_CONS_WARPS - 1) / C8_CONS_WARPS)   /* items per warp and tile */
// a stage: the span slots of four sub-vectors (sum_i m_i (16 alpha_i + 8) <=
// 4 * 315 * 16 + 8 * 248 words), then each span's alignment lead
#define C8_SDW (4 * C8_L * C8_T + C8_SPAN_PAD * C8_MAXSPANS)
#define C8_SW (((C8_SDW + C8_MAXSPANS) + 31) & ~31)
// exchange: per consumer warp two slots of IPW items x 32 half-sums
#define C8_XW (C8_CONS_WARPS * 2 * C8_IPW * 32)
// common area: J[L + 1], lane table [4][L], per span its start, slot and sub-vector
#define C8_CW ((C8_L + 1) + 4 * C8_L + 3 * C8_MAXSPANS)
#define C8_SMEM_BYTES (4 * (C8_STAGES * C8_SW + C8_XW + C8_CW))

static_assert(C8_SMEM_BYTES <= 227 * 1024 - 2048, "stage ring exceeds shared memory");
static_assert((C8_SW * 4) % 128 == 0, "stages must stay 128-byte aligned");
static_assert(32 * C8_PROD_WARPS * C8_KS >= C8_MAXSPANS, "producer threads cannot hold every span");
static_assert(C8_IPW % 4 == 0, "half-sums travel in groups of four");

namespace {

using namespace wl_tma;

__device__ __forceinline__ uint32_t c8_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}

// address of the same shared-memory word in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t c8_mapa(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

// 16 bytes into the partner's shared memory, counted as transaction bytes on
// the partner's mbarrier `rbar` when they land (no fence in this thread: a
// release at cluster scope would first wait for every global store this
// thread still has in flight)
__device__ __forceinline__ void c8_st_async4(uint32_t raddr, float a, float b, float c, float d, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];\n" ::"r"(
                     raddr),
                 "f"(a), "f"(b), "f"(c), "f"(d), "r"(rbar)
                 : "memory");
}

__device__ __forceinline__ void c8_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

// bounded wait on a local mbarrier phase, acquiring at cluster scope the
// partner's stores counted on it
__device__ __forceinline__ bool c8_wait_cluster(uint32_t bar, uint32_t parity)
{
    const long long start = clock64();
    while (true) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
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

__device__ __forceinline__ void c8_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}


__device__ __forceinline__ float c8_wait_prev(WlDevState *st, volatile float *s_c)
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
__global__ void __launch_bounds__(C8_THREADS, 1) tma8c_kernel(WlPassArgs a, double rnu)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar_full[C8_STAGES];
    __shared__ __align__(8) uint64_t bar_empty[C8_STAGES];
    // per consumer warp and exchange slot: the partner warp's half-sums are here
    __shared__ __align__(8) uint64_t bar_x[C8_CONS_WARPS][2];
    __shared__ uint64_t red[3 * (C8_THREADS / 32 + 1)];
    __shared__ volatile int s_abort;
    __shared__ int64_t s_gam[8];
    __shared__ int s_alpha[8];
    __shared__ uint32_t s_signs;
    __shared__ volatile float s_c;

    WlDevState *st = a.st;
    const float *__restrict__ src = (const float *)a.src;
    float *__restrict__ dst = (float *)a.dst;
    const int64_t N = a.N, Np = a.Np;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rank = (int)c8_rank();          // this CTA's half: sub-vectors 4 rank .. 4 rank + 3
    const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
    if (warp == 0) {
        const WlStrides *cur = &st->ahead[a.pass & 1];
        if (lane < 8)
            s_alpha[lane] = __ldcg(&cur->alpha[lane]);
        else if (lane < 16)
            s_gam[lane - 8] = (int64_t)__ldcg((const long long *)&cur->gamma[lane - 8]);
        else if (lane == 16)
            s_signs = SG ? __ldcg(&cur->signs) : 0u;
    }
    if (tid == 0) {
        for (int s = 0; s < C8_STAGES; s++) {
            mbar_init(smem_u32(&bar_full[s]), 32 * C8_PROD_WARPS);
            mbar_init(smem_u32(&bar_empty[s]), C8_CONS_WARPS);
        }
        for (int w = 0; w < C8_CONS_WARPS; w++) {
            mbar_init(smem_u32(&bar_x[w][0]), 1);
            mbar_init(smem_u32(&bar_x[w][1]), 1);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    // both CTAs' barriers are initialised before either arrives remotely
    c8_cluster_sync();
    const uint32_t signs = SG ? s_signs : 0u;

    // the same test as the one-CTA kernel, on all eight strides (both CTAs
    // of a cluster decide alike)
    bool tileable = true;
    int e3 = 0, e5 = 0, e7 = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int al = s_alpha[i];
        tileable &= al > 1 && al <= C8_L && C8_L % al == 0;
        e3 = max(e3, al % 9 == 0 ? 2 : (al % 3 == 0 ? 1 : 0));
        e5 |= al % 5 == 0 ? 1 : 0;
        e7 |= al % 7 == 0 ? 1 : 0;
    }
    tileable &= e3 == 2 && e5 == 1 && e7 == 1;
    // this CTA's four sub-vectors
    int alpha[4], m[4], sb[5];
    sb[0] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        alpha[i] = s_alpha[4 * rank + i];
        m[i] = tileable ? C8_L / alpha[i] : 0;
        sb[i + 1] = sb[i] + m[i];
    }
    const int nspans = sb[4];

    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    float *out = (float *)a.out;
    const float mu = (float)a.mu, sigma = (float)a.sigma;
    const int64_t w0 = a.w0, w1 = a.w1;
    float c;

    if (!tileable || nspans > C8_MAXSPANS || N < TM_MIN_N || (N & 3)) {
        // plain strided gather for this pass: every CTA on its own share of
        // j, all eight sub-vectors, no exchange
        c = c8_wait_prev(st, &s_c);
        const int64_t G = (int64_t)gridDim.x * blockDim.x;
        for (int64_t j = (int64_t)blockIdx.x * blockDim.x + tid; j < N; j += G) {
            float g[8], y[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int64_t ix = (int64_t)(((uint64_t)s_alpha[i] * (uint64_t)j + (uint64_t)s_gam[i]) % (uint64_t)N);
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
        float *xbuf = smem + C8_STAGES * C8_SW;   // [warp][slot][item][32]: the partner's half-sums
        int *common = (int *)(xbuf + C8_XW);
        int *J = common;                          // [L + 1] lane starts
        int *lanetab = J + (C8_L + 1);            // [4][L]: slot word of the lane's first value << 9 | span
        int *spanC = lanetab + 4 * C8_L;          // [spans]: ceil(p N / m_i)
        int *spanOff = spanC + C8_MAXSPANS;       // [spans]: slot offset in a stage, words
        int *spanSub = spanOff + C8_MAXSPANS;     // [spans]: sub-vector 0..3 of this CTA
        int slot0[4];
        slot0[0] = 0;
#pragma unroll
        for (int i = 0; i < 3; i++)
            slot0[i + 1] = slot0[i] + m[i] * (C8_T * alpha[i] + C8_SPAN_PAD);

        // ceil(l N / L) as l (N / L) + ceil(l (N mod L) / L), 32-bit (N <= 2^28)
        const int N32 = (int)N;
        {
            const int qL = N32 / C8_L, rL = N32 - qL * C8_L;
            for (int l = tid; l <= C8_L; l += C8_THREADS)
                J[l] = l * qL + (l * rL + C8_L - 1) / C8_L;
        }
        for (int sp = tid; sp < nspans; sp += C8_THREADS) {
            int i = 0, p = 0, mi = 1, al = 1, so = 0;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (sp >= sb[k] && sp < sb[k + 1]) {
                    i = k;
                    p = sp - sb[k];
                    mi = m[k];
                    al = alpha[k];
                    so = slot0[k];
                }
            const int qN = N32 / mi, rN = N32 - qN * mi;
            spanC[sp] = p * qN + (p * rN + mi - 1) / mi;
            spanOff[sp] = so + p * (C8_T * al + C8_SPAN_PAD);
            spanSub[sp] = i;
        }
        __syncthreads();
        // lane l of sub-vector i reads span p = l mod m_i from offset
        // r = alpha_i J_l - floor(l / m_i) N - spanC in [0, alpha_i)
        for (int e = tid; e < 4 * C8_L; e += C8_THREADS) {
            const int i = e / C8_L, l = e - i * C8_L;
            int mi = 1, al = 1, s0 = 0;
#pragma unroll
            for (int k = 0; k < 4; k++)
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
        c = c8_wait_prev(st, &s_c);
        const int maxlen = (N32 + C8_L - 1) / C8_L;
        const int ntiles = (maxlen + C8_T - 1) / C8_T;

        if (warp >= C8_CONS_WARPS) {
            // ---------------- producer warps ----------------
            // tiles cid, cid + C, ... (C clusters); both CTAs take the same
            const int pw = warp - C8_CONS_WARPS;
            const int pt = pw + C8_PROD_WARPS * lane;   // spans pt + 32 PW q, q < KS
            const uint32_t stage_base = smem_u32(stage0);
            int issued0 = 0, issued1 = 0;   // per stage: uses issued (phase parity of the last)
            for (int it = 0;; it++) {
                const int s = it & 1, k = it >> 1;
                const int tile = cid + it * ncl;
                if (tile >= ntiles || s_abort)
                    break;
                if (k > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (uint32_t)((k - 1) & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const uint32_t full = smem_u32(&bar_full[s]);
                const int t0 = tile * C8_T;
                const int Tt = min(C8_T, maxlen - t0);
                int *lead = (int *)(stage0 + s * C8_SW + C8_SDW);
                const uint32_t sbase = stage_base + 4u * (uint32_t)(s * C8_SW);
                int sa[C8_KS], sl[C8_KS], sub[C8_KS], soff[C8_KS];
                uint32_t total = 0;
#pragma unroll
                for (int q = 0; q < C8_KS; q++) {
                    const int sp = pt + 32 * C8_PROD_WARPS * q;
                    sl[q] = 0;
                    sa[q] = 0;
                    sub[q] = 0;
                    soff[q] = 0;
                    if (sp < nspans) {
                        const int i = spanSub[sp];
                        const int al = s_alpha[4 * rank + i];
                        int64_t ad = (int64_t)spanC[sp] + (int64_t)al * t0 + s_gam[4 * rank + i];   // < 3N
                        if (ad >= N)
                            ad -= N;
                        if (ad >= N)
                            ad -= N;
                        sa[q] = (int)ad;
                        sl[q] = al * Tt;
                        sub[q] = 4 * rank + i;
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
                for (int q = 0; q < C8_KS; q++) {
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
            uint32_t all_ret = 0, part_ret = 0;   // this CTA's rows returned whole, in part
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int64_t q0 = (4 * rank + i) * N, q1 = q0 + N;
                if (q1 > w0 && q0 < w1) {
                    if (q0 >= w0 && q1 <= w1)
                        all_ret |= 1u << i;
                    else
                        part_ret |= 1u << i;
                }
            }
            float *drow = dst + (int64_t)(4 * rank) * Np;
            const int64_t qrow = (int64_t)(4 * rank) * N - w0;   // out index of row 4 rank, j = 0
            const int ll = lane >> 4, tt = lane & 15;   // lane of the item, lane time
            const uint32_t xpart = c8_mapa(smem_u32(xbuf), (uint32_t)(rank ^ 1));
            const uint32_t bxpart = c8_mapa(smem_u32(&bar_x[warp][0]), (uint32_t)(rank ^ 1));
            const uint32_t bxown = smem_u32(&bar_x[warp][0]);
            uint32_t emax = 0;
            for (int it = 0;; it++) {
                const int s = it & 1, k = it >> 1;
                const int tile = cid + it * ncl;
                if (tile >= ntiles || s_abort)
                    break;
                if (!mbar_wait(smem_u32(&bar_full[s]), (uint32_t)(k & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int t0 = tile * C8_T;
                const int Tt = min(C8_T, maxlen - t0);
                const float *sdata = stage0 + s * C8_SW;
                const int *lead = (const int *)(sdata + C8_SDW);
                // item g of tile k goes to warp (k groups + g) mod C8_CONS_WARPS,
                // in both CTAs alike
                int g0 = warp - (int)(((uint32_t)tile * (uint32_t)C8_GROUPS) % C8_CONS_WARPS);
                g0 += g0 < 0 ? C8_CONS_WARPS : 0;
                // phase 1: this CTA's four values of every tuple and their sum
                float xv[C8_IPW][4];
                uint32_t ok = 0;
                // slot layout: [u / 4][thread][u mod 4], 16 bytes per thread and group
                const uint32_t xslot = xpart + 4u * (uint32_t)(((warp * 2 + (it & 1)) * C8_IPW) * 32 + 4 * lane);
                const uint32_t xbar = bxpart + 8u * (uint32_t)(it & 1);
                float hq[4];
#pragma unroll
                for (int u = 0; u < C8_IPW; u++) {
                    const int g = g0 + u * C8_CONS_WARPS;
                    const int l = 2 * g + ll;
                    float hs = 0.0f;
                    if (g < C8_GROUPS && l < C8_L) {
                        const int jl = J[l];
                        if (tt < min(Tt, J[l + 1] - jl - t0)) {
                            ok |= 1u << u;
#pragma unroll
                            for (int i = 0; i < 4; i++) {
                                const int lb = lanetab[i * C8_L + l];
                                float x = sdata[(lb >> 9) + lead[lb & 511] + alpha[i] * tt];
                                if (SG)   // the pass's matrix is A D_k
                                    x = wl_sgn(x, signs, 4 * rank + i);
                                xv[u][i] = x;
                            }
                            hs = __fadd_rn(__fadd_rn(xv[u][0], xv[u][1]), __fadd_rn(xv[u][2], xv[u][3]));
                        }
                    }
                    hq[u & 3] = hs;
                    if ((u & 3) == 3)   // every group is sent, used or not: 1 KB per warp and tile
                        c8_st_async4(xslot + 512u * (uint32_t)(u >> 2), hq[0], hq[1], hq[2], hq[3], xbar);
                }
                // stage free; expect the partner warp's 1 KB of half-sums
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&bar_empty[s]));
                    c8_arrive_expect_tx(bxown + 8u * (uint32_t)(it & 1), 32u * 4u * C8_IPW);
                }
                if (!c8_wait_cluster(bxown + 8u * (uint32_t)(it & 1), (uint32_t)((it >> 1) & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                // phase 2: h = (ab + de) / 4 and this CTA's four outputs
                const float *xown = xbuf + ((warp * 2 + (it & 1)) * C8_IPW) * 32 + 4 * lane;
                float4 xo;
                uint64_t tl = 0;   // at most 8 items x 4 terms per thread, each below 2^48
#pragma unroll
                for (int u = 0; u < C8_IPW; u++) {
                    if ((u & 3) == 0)   // the partner's half-sums of items u .. u + 3
                        xo = *(const float4 *)(xown + 128 * (u >> 2));
                    if (!((ok >> u) & 1u))
                        continue;
                    // this CTA's half-sum again (three adds instead of a register per item)
                    const float hs = __fadd_rn(__fadd_rn(xv[u][0], xv[u][1]), __fadd_rn(xv[u][2], xv[u][3]));
                    const float o = (u & 3) == 0 ? xo.x : (u & 3) == 1 ? xo.y : (u & 3) == 2 ? xo.z : xo.w;
                    const float h = __fmul_rn(__fadd_rn(hs, o), 0.25f);
                    const int j = J[2 * (g0 + u * C8_CONS_WARPS) + ll] + t0 + tt;
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float y = __fmul_rn(__fsub_rn(h, xv[u][i]), c);
                        drow[i * Np + j] = y;
                        tl += term32(y, emax);
                        const int64_t q = qrow + i * N + j;   // out index
                        if ((all_ret >> i) & 1u)
                            out[q] = __fadd_rn(mu, __fmul_rn(sigma, y));
                        else if (((part_ret >> i) & 1u) && q >= 0 && q < w1 - w0)
                            out[q] = __fadd_rn(mu, __fmul_rn(sigma, y));
                    }
                }
                lo += tl;
                hi += lo < tl ? 1ull : 0ull;
            }
            bad = emax >= 135u ? 1u : 0u;
        }
    }

    // no partner store or arrival can follow this point: both CTAs stay
    // resident until each has passed it
    c8_cluster_sync();
    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st))
        wl_finalise_cta(st, 8, N, a.nu, rnu, &dst[wl_last_phys(8, N, Np)], SG ? 1 : 0);
}

bool g_tma8c_configured[2] = {false, false};
int g_tma8c_clusters[2] = {0, 0};

} // namespace

// Set the kernel's shared-memory size once and find how many clusters of
// two can be resident at once (0 when none can: the kernel is then not used).
static int c8_configure(int which)
{
    if (g_tma8c_configured[which])
        return g_tma8c_clusters[which];
    auto kern = which ? tma8c_kernel<true> : tma8c_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C8_SMEM_BYTES) != cudaSuccess) {
        cudaGetLastError();
        g_tma8c_configured[which] = true;
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(C8_THREADS);
    cfg.dynamicSmemBytes = C8_SMEM_BYTES;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nc = 0;
    }
    g_tma8c_clusters[which] = nc;
    g_tma8c_configured[which] = true;
    return nc;
}

bool wl_tma8c_supported(int n, int64_t N, int fp64)
{
    return wl_tma8_supported(n, N, fp64) && c8_configure(0) > 0 && c8_configure(1) > 0;
}

int wl_tma8c_grid()
{
    return 2 * min(c8_configure(0), c8_configure(1));
}

cudaError_t wl_launch_tma8c(const WlPassArgs &a, int sm_count, int signs, cudaStream_t stream)
{
    const int which = signs ? 1 : 0;
    const int nc = c8_configure(which);
    if (nc <= 0)
        return cudaErrorNotSupported;
    auto kern = which ? tma8c_kernel<true> : tma8c_kernel<false>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * nc);   // every cluster resident: tiles are dealt statically
    cfg.blockDim = dim3(C8_THREADS);
    cfg.dynamicSmemBytes = C8_SMEM_BYTES;
    cfg.stream = stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    const double rnu = sqrt(2.0 * (double)a.nu - 1.0);   // IEEE square root: correctly rounded
    // large pools: the returned values follow in the streaming kernel
    const bool split = wl_tma8_return_kernel(a);
    WlPassArgs p = a;
    if (split)
        p.w0 = p.w1 = 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, p, rnu);
    if (e != cudaSuccess || !split)
        return e != cudaSuccess ? e : cudaGetLastError();
    return wl_launch_t8_return(a, sm_count, stream);
}
