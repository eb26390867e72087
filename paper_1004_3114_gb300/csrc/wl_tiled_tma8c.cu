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
// Tiles come from the generator's counter, one at a time, as in the one-CTA
// kernel (clusters sweep neighbouring tiles together, which keeps the half
// sectors at the ends of a lane's runs in L2 until their neighbours arrive;
// a static deal let the clusters drift apart, and partial sectors then went
// to DRAM as read-modify-writes).  CTA 0's producer draws the tile for ring
// slot q = k mod 4 once its stage is free and sends the index to both CTAs
// (4-byte st.async counted on each CTA's slot barrier, whose expected bytes
// each CTA's producer posts).  Slot q is written again only for iteration
// k + 4, after every warp of CTA 1 has passed iteration k + 1 (the half-sum
// exchange keeps the CTAs' warps within one tile of each other).  The sum of
// squares goes to the generator's accumulators from both CTAs and the last
// CTA of the grid (by ticket) runs the end of pass, as in the other pass
// kernels.  Every wait
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
#define C8_CONS_WARPS 16          /* 20 warps in all: 96 registers a thread (24: 80, spilling) */
#define C8_PROD_WARPS 4
#define C8_KS ((C8_MAXSPANS + 32 * C8_PROD_WARPS - 1) / (32 * C8_PROD_WARPS))
#define C8_THREADS (32 * (C8_CONS_WARPS + C8_PROD_WARPS))
// consumer items: 4 lanes x 16 lane times, a thread taking lane times t and
// t + 8 of one lane (one table read for both)
#define C8_ITEMS ((C8_L + 3) / 4)
#define C8_IPW ((C8_ITEMS + C8_CONS_WARPS - 1) / C8_CONS_WARPS)   /* items per warp and tile */
#define C8_TPT (2 * C8_IPW)      /* tuples per thread and tile */
// a stage: the span slots of four sub-vectors, sum_i m_i (16 alpha_i + 8) <=
// 4 * 315 * 16 + 8 * 248 words
#define C8_SDW (4 * C8_L * C8_T + C8_SPAN_PAD * C8_MAXSPANS)
#define C8_SW ((C8_SDW + 31) & ~31)
// exchange: per consumer warp two slots of C8_TPT half-sums per thread
#define C8_XW (C8_CONS_WARPS * 2 * C8_TPT * 32)
// common area: J[L + 1], lane table [4][L], per span its start, slot and sub-vector
#define C8_CW ((C8_L + 1) + 4 * C8_L + 3 * C8_MAXSPANS)
#define C8_SMEM_BYTES (4 * (C8_STAGES * C8_SW + C8_XW + C8_CW))

static_assert(C8_SMEM_BYTES <= 227 * 1024 - 2048, "stage ring exceeds shared memory");
static_assert((C8_SW * 4) % 128 == 0, "stages must stay 128-byte aligned");
static_assert(32 * C8_PROD_WARPS * C8_KS >= C8_MAXSPANS, "producer threads cannot hold every span");
static_assert(C8_T == 16, "a half-warp takes a lane's 16 lane times");
#define T8C_PREFER_BYTES (64ll << 20)

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

// 8 bytes into the partner's shared memory, counted as transaction bytes on
// the partner's mbarrier `rbar` when they land (no fence in this thread: a
// release at cluster scope would first wait for every global store this
// thread still has in flight)
__device__ __forceinline__ void c8_st_async2(uint32_t raddr, float a, float b, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];\n" ::"r"(raddr),
                 "f"(a), "f"(b), "r"(rbar)
                 : "memory");
}

__device__ __forceinline__ void c8_st_async1(uint32_t raddr, int v, uint32_t rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];\n" ::"r"(raddr), "r"(v),
                 "r"(rbar)
                 : "memory");
}

// the expected bytes of the partner's half-sums: orders nothing of this
// thread's, so relaxed
__device__ __forceinline__ void c8_arrive_expect_tx_relaxed(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(
                     bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void c8_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

#define C8_SUSPEND_NS 20000u   /* longest suspension of one try_wait */

// one try_wait on a phase of a local mbarrier; CL: acquire at cluster scope
// (what the partner CTA's stores counted on it wrote), else at CTA scope
template <bool CL>
__device__ __forceinline__ bool c8_try(uint32_t bar, uint32_t parity, uint32_t ns)
{
    uint32_t done;
    if (CL)
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity), "r"(ns)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity), "r"(ns)
                     : "memory");
    return done != 0;
}

// whether a phase of a local mbarrier has completed, without waiting
template <bool CL>
__device__ __forceinline__ bool c8_test(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    if (CL)
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
    return done != 0;
}

// bounded wait on a phase of a local mbarrier: true once it has completed,
// false after about a second.  A phase already complete costs one try_wait;
// otherwise each try_wait may suspend the thread until the phase completes.
template <bool CL>
__device__ __forceinline__ bool c8_wait(uint32_t bar, uint32_t parity)
{
    if (c8_test<CL>(bar, parity))
        return true;
    const long long start = clock64();
    while (!c8_try<CL>(bar, parity, C8_SUSPEND_NS))
        if (clock64() - start > TM_WAIT_CYCLES)
            return false;
    return true;
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

// SG: the generator draws a sign pattern each pass (matrix A D_k).  RET: the
// pass writes returned values (pools up to 64 MB; larger ones leave them to
// the streaming kernel), so passes without them carry none of their index
// arithmetic.
template <bool SG, bool RET>
__global__ void __launch_bounds__(C8_THREADS, 1) tma8c_kernel(WlPassArgs a, double rnu)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar_full[C8_STAGES];
    __shared__ __align__(8) uint64_t bar_empty[C8_STAGES];
    // per consumer warp and exchange slot: the partner warp's half-sums are here
    __shared__ __align__(8) uint64_t bar_x[C8_CONS_WARPS][2];
    // the tile of ring slot q (iterations q, q + 4, ...), drawn by CTA 0 of the cluster
    __shared__ __align__(8) uint64_t bar_tile[4];
    __shared__ volatile int s_tile[4];
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
        for (int q = 0; q < 4; q++)
            mbar_init(smem_u32(&bar_tile[q]), 1);
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
        float *xbuf = smem + C8_STAGES * C8_SW;   // [warp][slot][group][thread][4]: the partner's half-sums
        int *common = (int *)(xbuf + C8_XW);
        int *J = common;                          // [L + 1] lane starts
        int *offt = J + (C8_L + 1);               // [4][L]: stage word of the lane's first value
        int *spanC = offt + 4 * C8_L;             // [spans]: ceil(p N / m_i)
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
        // r = alpha_i J_l - floor(l / m_i) N - spanC in [0, alpha_i), after
        // the span's alignment lead: the copy of the span of tile k starts at
        // s = (spanC + alpha_i 16 k + gamma_i) mod N rounded down to a multiple
        // of 4, and with 16 k and N multiples of 4 its lead s mod 4 =
        // (spanC + gamma_i) mod 4 is the same in every tile
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
            const int lead = (int)(((int64_t)spanC[sp] + s_gam[4 * rank + i]) & 3);
            offt[e] = spanOff[sp] + lead + (int)r;
        }
        __syncthreads();
        c = c8_wait_prev(st, &s_c);
        const int maxlen = (N32 + C8_L - 1) / C8_L;
        const int minlen = N32 / C8_L;   // every lane has minlen or maxlen lane times
        const int ntiles = (maxlen + C8_T - 1) / C8_T;

        if (warp >= C8_CONS_WARPS) {
            // ---------------- producer warps ----------------
            const int pw = warp - C8_CONS_WARPS;
            const int pt = pw + C8_PROD_WARPS * lane;   // spans pt + 32 PW q, q < KS
            const uint32_t stage_base = smem_u32(stage0);
            int issued0 = 0, issued1 = 0;   // per stage: uses issued (phase parity of the last)
            for (int it = 0;; it++) {
                const int s = it & 1, k = it >> 1, ts = it & 3;
                if (s_abort)
                    break;
                if (k > 0 && !c8_wait<false>(smem_u32(&bar_empty[s]), (uint32_t)((k - 1) & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                // the stage is free in this CTA: CTA 0 draws the next tile from
                // the generator's counter and sends it to both CTAs
                if (pw == 0 && lane == 0) {
                    c8_arrive_expect_tx(smem_u32(&bar_tile[ts]), 4u);
                    if (rank == 0) {
                        const int t = (int)atomicAdd(&st->tile_ctr, 1u);
                        const uint32_t a_t = smem_u32((const void *)&s_tile[ts]), a_b = smem_u32(&bar_tile[ts]);
                        c8_st_async1(c8_mapa(a_t, 0u), t, c8_mapa(a_b, 0u));
                        c8_st_async1(c8_mapa(a_t, 1u), t, c8_mapa(a_b, 1u));
                    }
                }
                if (!c8_wait<true>(smem_u32(&bar_tile[ts]), (uint32_t)((it >> 2) & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int tile = s_tile[ts];
                if (tile >= ntiles)
                    break;
                const uint32_t full = smem_u32(&bar_full[s]);
                const int t0 = tile * C8_T;
                const int Tt = min(C8_T, maxlen - t0);
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
            if (issued0 > 0 && !c8_wait<false>(smem_u32(&bar_full[0]), (uint32_t)((issued0 - 1) & 1)))
                atomicOr(&st->status, WL_ETIMEOUT);
            if (issued1 > 0 && !c8_wait<false>(smem_u32(&bar_full[1]), (uint32_t)((issued1 - 1) & 1)))
                atomicOr(&st->status, WL_ETIMEOUT);
        } else {
            // ---------------- consumer warps ----------------
            // a thread's two tuples: lane time tt of lanes 4 g + ll and
            // 4 g + 2 + ll of item g (a half-warp stores a lane's 16 values:
            // 64 contiguous bytes per row)
            const int ll = lane >> 4, tt = lane & 15;
            int at[4];
#pragma unroll
            for (int i = 0; i < 4; i++)
                at[i] = alpha[i] * tt;
            float *drow = dst + (int64_t)(4 * rank) * Np;
            const int64_t qrow = (int64_t)(4 * rank) * N - w0, W = w1 - w0;   // out index of row 4 rank, j = 0
            const uint32_t xpart = c8_mapa(smem_u32(xbuf), (uint32_t)(rank ^ 1));
            const uint32_t bxpart = c8_mapa(smem_u32(&bar_x[warp][0]), (uint32_t)(rank ^ 1));
            const uint32_t bxown = smem_u32(&bar_x[warp][0]);
            uint32_t emax = 0;
            for (int it = 0;; it++) {
                const int s = it & 1, k = it >> 1, par = it & 1;
                if (s_abort)
                    break;
                if (!c8_wait<true>(smem_u32(&bar_tile[it & 3]), (uint32_t)((it >> 2) & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int tile = s_tile[it & 3];
                if (tile >= ntiles)
                    break;
                if (!c8_wait<false>(smem_u32(&bar_full[s]), (uint32_t)(k & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                const int t0 = tile * C8_T;
                const int Tt = min(C8_T, maxlen - t0);
                const bool full = t0 + C8_T <= minlen;   // every tuple of the tile exists
                const float *sdata = stage0 + s * C8_SW;
                // item g of tile k goes to warp (k items + g) mod C8_CONS_WARPS,
                // in both CTAs alike
                int g0 = warp - (int)(((uint32_t)tile * (uint32_t)C8_ITEMS) % C8_CONS_WARPS);
                g0 += g0 < 0 ? C8_CONS_WARPS : 0;
                // which tuples exist: items past the last, the lane past L in
                // the last item and, in the last tiles, lane times past a
                // lane's end; lanes past L read lane L - 1 (unused), so the
                // loads below need no branch
                int lcs[C8_TPT];   // lane of tuple v = 2 u + h
                uint32_t ok = 0;
#pragma unroll
                for (int v = 0; v < C8_TPT; v++) {
                    const int g = g0 + (v >> 1) * C8_CONS_WARPS;
                    const int l = 4 * g + 2 * (v & 1) + ll;
                    lcs[v] = min(l, C8_L - 1);
                    ok |= (g < C8_ITEMS && l < C8_L ? 1u : 0u) << v;
                }
                if (!full) {
#pragma unroll
                    for (int v = 0; v < C8_TPT; v++) {
                        const int lim = min(Tt, J[lcs[v] + 1] - J[lcs[v]] - t0);
                        ok &= ~((tt < lim ? 0u : 1u) << v);
                    }
                }
                // phase 1: this CTA's four values of each tuple and their sum
                float x0[C8_IPW][4], x1[C8_IPW][4];
                // slot layout: [item][thread][2], the thread's two tuples
                const uint32_t xslot = xpart + 4u * (uint32_t)((warp * 2 + par) * C8_TPT * 32 + 2 * lane);
                const uint32_t xbar = bxpart + 8u * (uint32_t)par;
#pragma unroll
                for (int u = 0; u < C8_IPW; u++) {
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        float v0 = sdata[offt[i * C8_L + lcs[2 * u]] + at[i]];
                        float v1 = sdata[offt[i * C8_L + lcs[2 * u + 1]] + at[i]];
                        if (SG) {   // the pass's matrix is A D_k
                            v0 = wl_sgn(v0, signs, 4 * rank + i);
                            v1 = wl_sgn(v1, signs, 4 * rank + i);
                        }
                        x0[u][i] = v0;
                        x1[u][i] = v1;
                    }
                }
#pragma unroll
                for (int u = 0; u < C8_IPW; u++)   // every item is sent, used or not: the slot's bytes per warp and tile
                    c8_st_async2(xslot + 256u * (uint32_t)u,
                                 __fadd_rn(__fadd_rn(x0[u][0], x0[u][1]), __fadd_rn(x0[u][2], x0[u][3])),
                                 __fadd_rn(__fadd_rn(x1[u][0], x1[u][1]), __fadd_rn(x1[u][2], x1[u][3])), xbar);
                // stage free; expect the partner warp's half-sums
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&bar_empty[s]));
                    c8_arrive_expect_tx_relaxed(bxown + 8u * (uint32_t)par, 4u * 32u * C8_TPT);
                }
                if (!c8_wait<true>(bxown + 8u * (uint32_t)par, (uint32_t)((it >> 1) & 1))) {
                    s_abort = 1;
                    atomicOr(&st->status, WL_ETIMEOUT);
                    break;
                }
                // phase 2: h = (ab + de) / 4 and this CTA's four outputs per tuple
                const float *xown = xbuf + (warp * 2 + par) * C8_TPT * 32 + 2 * lane;
                uint64_t tl = 0;   // at most 8 tuples x 4 terms per thread, each below 2^48
#pragma unroll
                for (int u = 0; u < C8_IPW; u++) {
                    const float2 xo = *(const float2 *)(xown + 64 * u);   // the partner's half-sums
                    const int j0 = J[lcs[2 * u]] + t0 + tt, j1 = J[lcs[2 * u + 1]] + t0 + tt;
                    const bool ok0 = (ok >> (2 * u)) & 1u, ok1 = (ok >> (2 * u + 1)) & 1u;
                    // this CTA's half-sums again (three adds instead of registers)
                    const float s0 = __fadd_rn(__fadd_rn(x0[u][0], x0[u][1]), __fadd_rn(x0[u][2], x0[u][3]));
                    const float s1 = __fadd_rn(__fadd_rn(x1[u][0], x1[u][1]), __fadd_rn(x1[u][2], x1[u][3]));
                    const float h0 = __fmul_rn(__fadd_rn(s0, xo.x), 0.25f);
                    const float h1 = __fmul_rn(__fadd_rn(s1, xo.y), 0.25f);
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float y0 = __fmul_rn(__fsub_rn(h0, x0[u][i]), c);
                        const float y1 = __fmul_rn(__fsub_rn(h1, x1[u][i]), c);
                        float *p = drow + i * Np;
                        if (ok0)
                            p[j0] = y0;
                        if (ok1)
                            p[j1] = y1;
                        // a missing tuple counts as 0 (term32(0) = 0, exponent 0)
                        tl += term32(ok0 ? y0 : 0.0f, emax);
                        tl += term32(ok1 ? y1 : 0.0f, emax);
                        if (RET) {
                            const int64_t q0 = qrow + i * N + j0, q1 = qrow + i * N + j1;   // out indices
                            if (ok0 && q0 >= 0 && q0 < W)
                                out[q0] = __fadd_rn(mu, __fmul_rn(sigma, y0));
                            if (ok1 && q1 >= 0 && q1 < W)
                                out[q1] = __fadd_rn(mu, __fmul_rn(sigma, y1));
                        }
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

bool g_tma8c_configured[4] = {false, false, false, false};
int g_tma8c_clusters[4] = {0, 0, 0, 0};

using C8Kernel = void (*)(WlPassArgs, double);

C8Kernel c8_kernel(int which)
{
    switch (which) {
    case 0:
        return tma8c_kernel<false, false>;
    case 1:
        return tma8c_kernel<false, true>;
    case 2:
        return tma8c_kernel<true, false>;
    default:
        return tma8c_kernel<true, true>;
    }
}

} // namespace

// Set the kernel's shared-memory size once and find how many clusters of
// two can be resident at once (0 when none can: the kernel is then not used).
// which = 2 signs + returned values in the pass.
static int c8_configure(int which)
{
    if (g_tma8c_configured[which])
        return g_tma8c_clusters[which];
    const C8Kernel kern = c8_kernel(which);
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
    if (!wl_tma8_supported(n, N, fp64))
        return false;
    for (int w = 0; w < 4; w++)
        if (c8_configure(w) <= 0)
            return false;
    return true;
}

bool wl_tma8c_preferred(int n, int64_t N, int fp64)
{
    // pools whose returned values go to the streaming kernel (over 64 MB):
    // there the cluster pass measured 2-10% faster than the one-CTA pass;
    // below, with the returned values in the pass, they tie
    return n == 8 && !fp64 && (int64_t)sizeof(float) * 8 * N > T8C_PREFER_BYTES;
}

int wl_tma8c_grid()
{
    int nc = c8_configure(0);
    for (int w = 1; w < 4; w++)
        nc = min(nc, c8_configure(w));
    return 2 * nc;
}

cudaError_t wl_launch_tma8c(const WlPassArgs &a, int sm_count, int signs, cudaStream_t stream)
{
    // large pools: the returned values follow in the streaming kernel
    const bool split = wl_tma8_return_kernel(a);
    WlPassArgs p = a;
    if (split)
        p.w0 = p.w1 = 0;
    const int which = (signs ? 2 : 0) + (p.w1 > p.w0 ? 1 : 0);
    const int nc = c8_configure(which);
    if (nc <= 0)
        return cudaErrorNotSupported;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * nc);   // every cluster resident
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, c8_kernel(which), p, rnu);
    if (e != cudaSuccess || !split)
        return e != cudaSuccess ? e : cudaGetLastError();
    return wl_launch_t8_return(a, sm_count, stream);
}
