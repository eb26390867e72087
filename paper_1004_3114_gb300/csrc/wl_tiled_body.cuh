// Per-CTA building blocks of one pass of a binary32, n = 4 Wallace generator
// (Eq. 1 of Brent's RANN4 paper), shared by the grid-wide lane-tiled kernel
// (wl_tiled.cu) and the batched kernel (wl_batch.cu):
//
//   wl_gather4_range -- plain strided gather over j = j0, j0 + step, ...; the
//                       index advances by alpha_i step mod N with one
//                       conditional subtraction (no modulo in the loop, as in
//                       the paper's vector loop of Section 7);
//   wl_tiled4_tiles  -- lane-tiled gather over a range of tiles.  With
//                       L = lcm(alpha_i) lanes starting at J_l = ceil(l N / L),
//                       a tile of T lane times reads, per sub-vector i,
//                       m_i = L / alpha_i contiguous spans of alpha_i T values
//                       (span p starts at ceil(p N / m_i) + alpha_i t0 +
//                       gamma_i mod N) and uses every value: 16-byte
//                       cp.async copies into shared memory, odd-stride
//                       (conflict-free) shared reads, unit-stride stores.
//
// Both accumulate the exact sum of squares of the values they produce and
// write the values with pool index in [w0, w1) to out[q - w0] as mu + sigma y.
#pragma once

#include "wl_common.cuh"

#define TL_LMAX 315
#define TL_MAXSPANS 420      /* sum_i L / alpha_i <= 4 * 315 / 3 */
#define TL_MAXWRAP 64
#define TL_EMAX 2560         /* lane-times per tile: L * T <= this */
#define TL_MIN_N_CTA 4096    /* N above the tile size: at most one wrapping span per sub-vector */

// One pass of one generator as seen by a CTA.
struct WlTileJob {
    const float *src;
    float *dst;
    int64_t N, Np;
    int alpha[4];
    int64_t gam[4];
    float c;
    float *out;
    int64_t w0, w1;
    float mu, sigma;
    uint32_t signs = 0;   // per-pass sign pattern (bit i negates g_i)
};

__host__ __device__ constexpr int tl_data_words() { return 4 * TL_EMAX + 4 * TL_MAXSPANS; }
__host__ __device__ constexpr int tl_int_words()
{
    return (TL_LMAX + 1) + 8 * TL_LMAX + 4 * TL_MAXSPANS + TL_MAXWRAP + 1;
}
__host__ __device__ constexpr size_t tl_smem_bytes()
{
    return sizeof(float) * (size_t)(tl_data_words() + tl_int_words());
}

__device__ __forceinline__ void tl_cp_async16(uint32_t saddr, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void tl_cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// floor(f / d) as umulhi(f, ceil(2^32 / d)): exact when f * d < 2^32 and d >= 2
// (the error f (ceil(2^32/d) - 2^32/d) / 2^32 < f / 2^32 < 1/d); d = 1 is passed through.
__device__ __forceinline__ uint32_t tl_magic(uint32_t d)
{
    // ceil(2^32 / d) = floor((2^32 - 1) / d) + 1 for d >= 2 (a 32-bit division)
    return d > 1 ? 0xffffffffu / d + 1u : 0u;
}
__device__ __forceinline__ uint32_t tl_div(uint32_t f, uint32_t d, uint32_t m)
{
    return d > 1 ? __umulhi(f, m) : f;
}

__device__ __forceinline__ int wl_lcm4(const int *alpha)
{
    // 32-bit gcd: strides and their lcm stay far below 2^31
    uint32_t L = (uint32_t)alpha[0];
#pragma unroll
    for (int i = 1; i < 4; i++) {
        uint32_t x = L, y = (uint32_t)alpha[i];
        while (y) {
            const uint32_t t = x % y;
            x = y;
            y = t;
        }
        L = L / x * (uint32_t)alpha[i];
    }
    return (int)L;
}

__device__ __forceinline__ bool wl_tiled_ok(int L, int64_t N)
{
    return L <= TL_LMAX && N >= TL_MIN_N_CTA && N <= ((int64_t)1 << 28);
}

// j_end < 0 means N
__device__ inline void wl_gather4_range(const WlTileJob &a, int64_t j, int64_t G, uint64_t &lo,
                                        uint64_t &hi, uint32_t &bad, int64_t j_end = -1)
{
    const int64_t N = a.N, Np = a.Np;
    const int64_t jmax = j_end < 0 ? N : j_end;
    int64_t idx[4], stp[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        idx[i] = (int64_t)(((uint64_t)a.alpha[i] * (uint64_t)(j < N ? j : 0) + (uint64_t)a.gam[i]) %
                           (uint64_t)N);
        stp[i] = (int64_t)(((uint64_t)a.alpha[i] * (uint64_t)G) % (uint64_t)N);
    }
    for (; j < jmax; j += G) {
        float g[4], y[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            g[i] = wl_sgn(a.src[i * Np + idx[i]], a.signs, i);
            idx[i] += stp[i];
            if (idx[i] >= N)
                idx[i] -= N;
        }
        wl_xform4(g, a.c, y);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            a.dst[k * Np + j] = y[k];
            wl_add128(lo, hi, wl_term32(y[k], bad), 0);
            const int64_t q = k * N + j;
            if (q >= a.w0 && q < a.w1)
                a.out[q - a.w0] = __fadd_rn(a.mu, __fmul_rn(a.sigma, y[k]));
        }
    }
}

// Every thread of the CTA must call this (it synchronises the CTA).  `smem`
// holds tl_smem_bytes() bytes, 16-byte aligned.  etarget <= TL_EMAX sets the
// tile size (L * T <= etarget, T a multiple of 4, at least 4).  With nparts
// > 1 only the tiles of part `part` (an even split of the pass's tiles into
// nparts ranges) are done.
__device__ inline void wl_tiled4_tiles(const WlTileJob &a, int L, int tile0, int tstep, int etarget,
                                       float *smem, uint64_t &lo, uint64_t &hi, uint32_t &bad,
                                       int part = 0, int nparts = 1)
{
    const int64_t N = a.N, Np = a.Np;
    const int tid = threadIdx.x, nth = blockDim.x;
    int m[4], sb[5], slot0[4], SL[4];
    int T = (etarget / L) & ~3;
    if (T < 4)
        T = 4;
    sb[0] = 0;
    slot0[0] = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        m[i] = L / a.alpha[i];
        SL[i] = a.alpha[i] * T + 4;   // copies cover at most alpha_i T + 4 values
        sb[i + 1] = sb[i] + m[i];
        if (i < 3)
            slot0[i + 1] = slot0[i] + m[i] * SL[i];
    }
    const int nspans = sb[4];
    int *J = (int *)(smem + tl_data_words());
    int *lanebase = J + (TL_LMAX + 1);
    int *laneoff = lanebase + 4 * TL_LMAX;
    int *spanC = laneoff + 4 * TL_LMAX;
    int *spanAs = spanC + TL_MAXSPANS;
    int *spanLead = spanAs + TL_MAXSPANS;
    int *spanAddr = spanLead + TL_MAXSPANS;
    int *s_wrap = spanAddr + TL_MAXSPANS;
    int *s_nwrap = s_wrap + TL_MAXWRAP;
    const uint32_t smem_base = (uint32_t)__cvta_generic_to_shared(smem);

    __syncthreads();   // the tables may still be read by a previous call
    // lane starts J_l = ceil(l N / L) and span bases C_ip = ceil(p N / m_i)
    for (int l = tid; l <= L; l += nth)
        J[l] = (int)(((int64_t)l * N + L - 1) / L);
    for (int s = tid; s < nspans; s += nth) {
        int i = (s >= sb[1]) + (s >= sb[2]) + (s >= sb[3]);
        int p = s - sb[i];
        spanC[s] = (int)(((int64_t)p * N + m[i] - 1) / m[i]);
    }
    __syncthreads();
    // lane l, sub-vector i: offset r in [0, alpha_i) inside its group's span
    for (int e = tid; e < 4 * L; e += nth) {
        int i = e / L, l = e - i * L;
        int w = l / m[i], p = l - w * m[i];
        int64_t r = (int64_t)a.alpha[i] * J[l] - (int64_t)w * N - spanC[sb[i] + p];
        lanebase[i * TL_LMAX + l] = slot0[i] + p * SL[i] + (int)r;
    }
    const int maxlen = (int)(((uint32_t)N + (uint32_t)L - 1u) / (uint32_t)L);
    const int ntiles_all = (maxlen + T - 1) / T;
    const int tbeg = (int)((int64_t)ntiles_all * part / nparts);
    const int ntiles = (int)((int64_t)ntiles_all * (part + 1) / nparts);
    __syncthreads();

    for (int tile = tbeg + tile0; tile < ntiles; tile += tstep) {
        const int t0 = tile * T;
        const int Tt = min(T, maxlen - t0);
        if (tid == 0)
            *s_nwrap = 0;
        __syncthreads();
        // where each span starts this tile; wrapping spans go to a list
        for (int s = tid; s < nspans; s += nth) {
            int i = (s >= sb[1]) + (s >= sb[2]) + (s >= sb[3]);
            int64_t addr = (int64_t)spanC[s] + (int64_t)a.alpha[i] * t0 + a.gam[i];
            while (addr >= N)
                addr -= N;
            int len = a.alpha[i] * Tt;
            spanAddr[s] = (int)addr;
            if (addr + len <= N) {
                int as = (int)addr & ~3;
                spanAs[s] = as;
                spanLead[s] = (int)addr - as;
            } else {
                spanAs[s] = -1;
                spanLead[s] = 0;
                int k = atomicAdd(s_nwrap, 1);
                if (k < TL_MAXWRAP)
                    s_wrap[k] = s;
            }
        }
        __syncthreads();
        // 16-byte copies of the aligned spans
#pragma unroll 1
        for (int i = 0; i < 4; i++) {
            const int K = (a.alpha[i] * Tt + 3) / 4 + 1;
            const uint32_t mk = tl_magic((uint32_t)K);
            const int total = m[i] * K;
            const float *srci = a.src + (int64_t)i * Np;
            for (int f = tid; f < total; f += nth) {
                int p = (int)tl_div((uint32_t)f, (uint32_t)K, mk);
                int ch = f - p * K;
                int as = spanAs[sb[i] + p];
                if (as >= 0)
                    tl_cp_async16(smem_base + 4u * (uint32_t)(slot0[i] + p * SL[i] + 4 * ch),
                                  srci + as + 4 * ch);
            }
        }
        // spans that run past the end of a sub-vector wrap to its start
        const int nw = min(*s_nwrap, TL_MAXWRAP);
        for (int k = 0; k < nw; k++) {
            int s = s_wrap[k];
            int i = (s >= sb[1]) + (s >= sb[2]) + (s >= sb[3]);
            int p = s - sb[i];
            int len = a.alpha[i] * Tt;
            int64_t addr = spanAddr[s];
            float *slot = smem + slot0[i] + p * SL[i];
            for (int u = tid; u < len; u += nth) {
                int64_t ad = addr + u;
                if (ad >= N)
                    ad -= N;
                slot[u] = a.src[(int64_t)i * Np + ad];
            }
        }
        // per-lane offsets for this tile
        for (int e = tid; e < 4 * L; e += nth) {
            int i = e / L, l = e - i * L;
            int p = l % m[i];
            laneoff[i * TL_LMAX + l] = lanebase[i * TL_LMAX + l] + spanLead[sb[i] + p];
        }
        tl_cp_async_wait_all();
        __syncthreads();
        // transform: pair f = (lane l, time t)
        const uint32_t mT = tl_magic((uint32_t)Tt);
        const int npairs = L * Tt;
        for (int f = tid; f < npairs; f += nth) {
            int l = (int)tl_div((uint32_t)f, (uint32_t)Tt, mT);
            int t = f - l * Tt;
            int jl = J[l];
            int tt = t0 + t;
            if (tt >= J[l + 1] - jl)
                continue;
            float g[4], y[4];
#pragma unroll
            for (int i = 0; i < 4; i++)
                g[i] = wl_sgn(smem[laneoff[i * TL_LMAX + l] + a.alpha[i] * t], a.signs, i);
            wl_xform4(g, a.c, y);
            const int64_t j = (int64_t)jl + tt;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                a.dst[k * Np + j] = y[k];
                wl_add128(lo, hi, wl_term32(y[k], bad), 0);
                const int64_t q = k * N + j;
                if (q >= a.w0 && q < a.w1)
                    a.out[q - a.w0] = __fadd_rn(a.mu, __fmul_rn(a.sigma, y[k]));
            }
        }
        __syncthreads();
    }
}
