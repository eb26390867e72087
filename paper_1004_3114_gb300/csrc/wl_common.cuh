// Device-side building blocks shared by the kernels of the Wallace generator
// (Brent, "A fast vectorised implementation of Wallace's normal random
// number generator", 1997): per-generator device state, the uniform source,
// per-pass parameter draw, sum-of-squares terms and reductions, and the
// end-of-pass finaliser (chi-squared rescale, Eq. 3, and drift monitor).
//
// Every floating-point operation whose result reaches the pool is written
// with an explicit IEEE round-to-nearest intrinsic (__fadd_rn, __dmul_rn, ...)
// so the compiler can neither contract nor reorder it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define WL_OK 0
#define WL_ECORRUPT 4
#define WL_ETIMEOUT 16

// Parameters of one pass (Eq. 1): strides alpha_i and offsets gamma_i, and
// the scale c folded into A (Section 4).
struct WlParams {
    int32_t alpha[8];
    int64_t gamma[8];
    float c32;
    uint32_t signs;     // bit i: sub-vector i negated before A (0 for the fixed A)
    double c64;
    // n = 2 (RANN4): the pass's rotation, and with the scale folded in
    // (C = c cos, S = c sin, rounded once to each precision)
    double rcos, rsin, rc64, rs64;
    float rc32, rs32;
};

// Strides and offsets of one pass.
struct WlStrides {
    int32_t alpha[8];
    int64_t gamma[8];
    uint32_t signs;
    uint32_t pad_;
    double rcos, rsin;   // n = 2: the pass's rotation
};

// One generator's device state.  The finaliser of a pass writes `next`;
// the following pass reads it.  The strides are drawn one pass ahead: with k
// passes completed, ahead[k & 1] holds pass k's (also in `next`) and
// ahead[(k + 1) & 1] pass k + 1's, so a kernel can read its own pass's
// strides before the previous pass has finished.  The uniform sequence is
// the same; `lcg_rep` is the state after the most recent pass's strides were
// drawn (after the initial pool before the first pass).  The accumulators are
// zero between passes.
struct WlDevState {
    WlParams next;          // parameters for the next pass
    WlParams last;          // parameters the most recent pass used
    WlStrides ahead[2];     // strides of passes k and k + 1, in slots k & 1 and (k + 1) & 1
    uint64_t lcg;           // uniform generator state (after the draw for pass k + 1)
    uint64_t lcg_pend;      // state before the draw for pass k + 1
    uint64_t lcg_rep;       // state before the draw for pass k (after the draw for pass k - 1)
    uint64_t acc0;          // running Q of the pass in flight, as three limbs that
    uint64_t acc1;          // CTAs add to without carries: bits 0-31, 32-63 and
    uint64_t acc2;          // 64-127 of each CTA's 128-bit sum (see wl_acc_read)
    uint32_t acc_bad;       // a value was non-finite or |y| >= 256
    uint32_t ticket;        // CTAs finished in the pass in flight
    uint64_t q_lo, q_hi;    // Q of the most recent pool
    double q, S, S_prev, c, drift;
    int32_t have_prev;
    int32_t status;         // sticky WL_* bits
    int32_t bad;
    int32_t chi;            // 0: Eq. 3's sample; 1: Wilson-Hilferty's (set at creation)
    int32_t msigns;         // 1: a random sign pattern per pass, matrix A D_k (set at creation)
    int32_t pad3_;
    int64_t passes;
    int32_t cand[11];       // n = 4, 8: the stride candidates for this N, increasing (set at creation)
    int32_t ncand;
    // next tile of the pass in flight (dynamically scheduled kernels): every
    // CTA takes tiles from it all pass long, so it has a cache line to itself
    alignas(128) uint32_t tile_ctr;
};

// ---- uniform source --------------------------------------------------------
// 64-bit LCG with Knuth's MMIX multiplier and increment, top 32 bits returned;
// seeded through SplitMix64 (Steele, Lea, Flood 2014) of (stream<<32 | seed).
#define WL_LCG_A 6364136223846793005ull
#define WL_LCG_C 1442695040888963407ull

__device__ __forceinline__ uint32_t wl_lcg_step(uint64_t &s)
{
    s = s * WL_LCG_A + WL_LCG_C;
    return (uint32_t)(s >> 32);
}

__device__ __forceinline__ uint64_t wl_seed_mix(uint32_t seed, uint32_t stream)
{
    uint64_t z = (((uint64_t)stream << 32) | (uint64_t)seed) + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// State after m steps, by composing the affine map s -> a s + c with itself
// (binary powering; F. B. Brown, "Random number generation with arbitrary
// strides", 1994).
__device__ __forceinline__ uint64_t wl_lcg_jump(uint64_t s, uint64_t m)
{
    uint64_t A = 1, C = 0, ap = WL_LCG_A, cp = WL_LCG_C;
    while (m) {
        if (m & 1) {
            A = ap * A;
            C = ap * C + cp;
        }
        cp = ap * cp + cp;
        ap = ap * ap;
        m >>= 1;
    }
    return A * s + C;
}

// ---- per-pass parameters ---------------------------------------------------
// Strides are distinct, odd, > 1 and coprime to N (Eq. 2, Sections 3 and 7).
// For n = 4 and 8 the candidates are the odd divisors > 1 of p^2 q (n = 4) or
// p^2 q r (n = 8), p < q < r the smallest odd primes not dividing N: all
// coprime to N, and one pass's strides have an lcm dividing p^2 q (p^2 q r),
// the lane count of the tiled kernels -- 45 (315) when N is coprime to 15
// (105).  One uniform per sub-vector picks, by multiply-shift, among the
// candidates not yet used, in increasing order.  n = 2 is RANN4 itself
// (Section 8): alpha from {3, 5} for x and beta from {7, 11} for y, those
// coprime to N; with none free, the smallest free odd number > 1 coprime to
// N.  The offset is floor(U N / 2^32), uniform on {0..N-1}.
// (32-bit remainders when both fit: a 64-bit remainder costs several hundred
// cycles on this part, a 32-bit one a few dozen)
__device__ __forceinline__ int64_t wl_gcd(int64_t a, int64_t b)
{
    if (((uint64_t)a | (uint64_t)b) >> 32 == 0) {
        uint32_t x = (uint32_t)a, y = (uint32_t)b;
        while (y) {
            const uint32_t t = x % y;
            x = y;
            y = t;
        }
        return (int64_t)x;
    }
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

__device__ __forceinline__ bool wl_stride_free(int32_t a, int64_t N, const int32_t *used, int k)
{
    if (wl_gcd(a, N) != 1)
        return false;
    for (int t = 0; t < k; t++)
        if (used[t] == a)
            return false;
    return true;
}

// The `need` smallest odd primes that do not divide N, from the odd primes
// below 64 (at most fourteen of them divide an N < 2^63).  N mod P in 32-bit
// arithmetic from N's halves (N = hi 2^32 + lo); N coprime to 15 takes two
// tests.  A rolled loop: the finaliser runs inside kernels that keep many
// registers live.
__device__ __forceinline__ void wl_free_primes(uint64_t uN, int need, uint32_t &p, uint32_t &q, uint32_t &r)
{
    constexpr uint32_t P[17] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61};
    const uint32_t hi = (uint32_t)(uN >> 32), lo = (uint32_t)uN;
    p = q = r = 0;
    int got = 0;
#pragma unroll 1
    for (int k = 0; k < 17; k++) {
        const uint32_t pk = P[k];
        const uint32_t r32 = (0xffffffffu % pk + 1u) % pk;   // 2^32 mod pk
        if (((hi % pk) * r32 + lo % pk) % pk != 0) {
            if (got == 0)
                p = P[k];
            else if (got == 1)
                q = P[k];
            else
                r = P[k];
            if (++got == need)
                break;
        }
    }
}

// The candidates for n = 4 (5 values) or n = 8 (11 values), increasing.
__device__ inline int wl_stride_candidates(int n, int64_t N, int32_t *cand)
{
    uint32_t p, q, r;
    wl_free_primes((uint64_t)N, n == 8 ? 3 : 2, p, q, r);
    int nc = 0;
    const int e3max = n == 8 ? 1 : 0;
    for (int e1 = 0; e1 <= 2; e1++) {
        const int32_t pe = e1 == 0 ? 1 : (e1 == 1 ? (int32_t)p : (int32_t)(p * p));
        for (int e2 = 0; e2 <= 1; e2++)
            for (int e3 = 0; e3 <= e3max; e3++) {
                const int32_t d = pe * (e2 ? (int32_t)q : 1) * (e3 ? (int32_t)r : 1);
                if (d > 1)
                    cand[nc++] = d;
            }
    }
    for (int a = 1; a < nc; a++) {
        const int32_t v = cand[a];
        int b = a - 1;
        while (b >= 0 && cand[b] > v) {
            cand[b + 1] = cand[b];
            b--;
        }
        cand[b + 1] = v;
    }
    return nc;
}

// n = 4 or 8 from NC = 5 or 11 candidates c (increasing) held in registers:
// a bit per candidate still free; sub-vector i takes the free candidate of
// rank floor(U k / 2^32) among the k free ones.
template <int NC>
__device__ __forceinline__ void wl_pick_strides(int64_t N, uint64_t &s, int32_t *alpha, int64_t *gamma,
                                                const int32_t (&c)[NC])
{
    constexpr int n = NC == 5 ? 4 : 8;
    uint32_t avail = (1u << NC) - 1u;
#pragma unroll(NC == 5 ? 4 : 1)
    for (int i = 0; i < n; i++) {
        const uint32_t u = wl_lcg_step(s);
        const uint32_t pick = (uint32_t)(((uint64_t)u * (uint64_t)__popc(avail)) >> 32);
        int32_t a = 0;
        uint32_t bit = 0, seen = 0;
#pragma unroll
        for (int b = 0; b < NC; b++) {
            const bool on = (avail >> b) & 1u;
            if (on && seen == pick) {
                a = c[b];
                bit = 1u << b;
            }
            seen += on ? 1u : 0u;
        }
        avail &= ~bit;
        alpha[i] = a;
        const uint32_t v = wl_lcg_step(s);
        gamma[i] = (int64_t)(((uint64_t)v * (uint64_t)N) >> 32);
    }
}

// ctab: the generator's candidates (wl_stride_candidates at creation); N
// coprime to 15 (n = 4) or 105 (n = 8) takes the same values as constants,
// so the finaliser of such pools reads no memory here.
__device__ inline void wl_draw_params(int n, int64_t N, uint64_t &s, int32_t *alpha, int64_t *gamma,
                                      const int32_t *ctab)
{
    const uint64_t uN = (uint64_t)N;
    const bool co15 = uN % 3u != 0 && uN % 5u != 0;
    if (n == 4) {
        int32_t c[5] = {3, 5, 9, 15, 45};
        if (!co15) {
#pragma unroll
            for (int k = 0; k < 5; k++)
                c[k] = ctab[k];
        }
        wl_pick_strides<5>(N, s, alpha, gamma, c);
        return;
    }
    if (n == 8) {
        int32_t c[11] = {3, 5, 7, 9, 15, 21, 35, 45, 63, 105, 315};
        if (!co15 || uN % 7u == 0) {
#pragma unroll
            for (int k = 0; k < 11; k++)
                c[k] = ctab[k];
        }
        wl_pick_strides<11>(N, s, alpha, gamma, c);
        return;
    }
    const int32_t rann4[2][2] = {{3, 5}, {7, 11}};
    for (int i = 0; i < n; i++) {
        const int32_t *cand = rann4[i];
        const uint32_t u = wl_lcg_step(s);
        int32_t freec[2];
        int nf = 0;
        for (int k = 0; k < 2; k++) {
            if (wl_gcd(cand[k], N) != 1)
                continue;
            bool used = false;
            for (int t = 0; t < i; t++)
                used |= alpha[t] == cand[k];
            if (!used)
                freec[nf++] = cand[k];
        }
        int32_t a;
        if (nf > 0) {
            a = freec[((uint64_t)u * (uint64_t)nf) >> 32];
        } else {
            a = 3;
            while (!wl_stride_free(a, N, alpha, i))
                a += 2;
        }
        alpha[i] = a;
        const uint32_t v = wl_lcg_step(s);
        gamma[i] = (int64_t)(((uint64_t)v * (uint64_t)N) >> 32);
    }
}

// ---- the transform (Section 2; A = (2/n)J - I, scaled by c) ----------------
// n = 2 (RANN4, Section 8): x' = C g0 + S g1, y' = C g1 - S g0 with the
// scale folded into the rotation (C = c cos theta, S = c sin theta).
__device__ __forceinline__ void wl_xform2(const float *g, float C, float S, float *y)
{
    y[0] = __fadd_rn(__fmul_rn(C, g[0]), __fmul_rn(S, g[1]));
    y[1] = __fsub_rn(__fmul_rn(C, g[1]), __fmul_rn(S, g[0]));
}

__device__ __forceinline__ void wl_xform2d(const double *g, double C, double S, double *y)
{
    y[0] = __dadd_rn(__dmul_rn(C, g[0]), __dmul_rn(S, g[1]));
    y[1] = __dsub_rn(__dmul_rn(C, g[1]), __dmul_rn(S, g[0]));
}

__device__ __forceinline__ void wl_xform4(const float *g, float c, float *y)
{
    float s = __fadd_rn(__fadd_rn(g[0], g[1]), __fadd_rn(g[2], g[3]));
    float h = __fmul_rn(s, 0.5f);
#pragma unroll
    for (int k = 0; k < 4; k++)
        y[k] = __fmul_rn(__fsub_rn(h, g[k]), c);
}

__device__ __forceinline__ void wl_xform8(const float *g, float c, float *y)
{
    float ab = __fadd_rn(__fadd_rn(g[0], g[1]), __fadd_rn(g[2], g[3]));
    float de = __fadd_rn(__fadd_rn(g[4], g[5]), __fadd_rn(g[6], g[7]));
    float h = __fmul_rn(__fadd_rn(ab, de), 0.25f);
#pragma unroll
    for (int k = 0; k < 8; k++)
        y[k] = __fmul_rn(__fsub_rn(h, g[k]), c);
}

__device__ __forceinline__ void wl_xform4d(const double *g, double c, double *y)
{
    double s = __dadd_rn(__dadd_rn(g[0], g[1]), __dadd_rn(g[2], g[3]));
    double h = __dmul_rn(s, 0.5);
#pragma unroll
    for (int k = 0; k < 4; k++)
        y[k] = __dmul_rn(__dsub_rn(h, g[k]), c);
}

__device__ __forceinline__ void wl_xform8d(const double *g, double c, double *y)
{
    double ab = __dadd_rn(__dadd_rn(g[0], g[1]), __dadd_rn(g[2], g[3]));
    double de = __dadd_rn(__dadd_rn(g[4], g[5]), __dadd_rn(g[6], g[7]));
    double h = __dmul_rn(__dadd_rn(ab, de), 0.25);
#pragma unroll
    for (int k = 0; k < 8; k++)
        y[k] = __dmul_rn(__dsub_rn(h, g[k]), c);
}

// ---- sum of squares (Section 4; Section 8 drift monitor) -------------------
// Binary32 pool: term = floor(y^2 2^32), computed exactly in integers from the
// significand m and exponent: y = m 2^(e-150) so y^2 2^32 = m^2 2^(2e-268).
// |y| >= 256 (exponent field >= 135, including Inf/NaN) flags the pool.
__device__ __forceinline__ uint64_t wl_term32(float y, uint32_t &bad)
{
    uint32_t u = __float_as_uint(y) & 0x7fffffffu;
    uint32_t e = u >> 23;
    bad |= (e >= 135u);
    uint32_t m = (u & 0x7fffffu) | (e ? 0x800000u : 0u);
    uint32_t ee = e ? e : 1u;
    uint32_t rs = 268u - 2u * ee;          // >= 0 for e <= 134
    uint64_t sq = (uint64_t)m * (uint64_t)m;
    uint64_t t = (rs < 64u) ? (sq >> rs) : 0ull;
    return (e >= 135u) ? 0ull : t;
}

// Binary64 pool: term = floor(fl(y*y) 2^64) as a 128-bit integer.
__device__ __forceinline__ void wl_term64(double y, uint64_t &lo, uint64_t &hi, uint32_t &bad)
{
    lo = 0;
    hi = 0;
    if (!(fabs(y) < 256.0)) {
        bad = 1;
        return;
    }
    double t = __dmul_rn(y, y);
    uint64_t u = (uint64_t)__double_as_longlong(t);
    int e = (int)((u >> 52) & 0x7ff);
    uint64_t m = (u & ((1ull << 52) - 1)) | (e ? (1ull << 52) : 0ull);
    int sh = (e ? e : 1) - 1075 + 64;      // t 2^64 = m 2^sh
    if (sh >= 0) {
        lo = m << sh;
        hi = sh ? (m >> (64 - sh)) : 0ull;
    } else if (sh > -64) {
        lo = m >> (-sh);
    }
}

__device__ __forceinline__ void wl_add128(uint64_t &lo, uint64_t &hi, uint64_t alo, uint64_t ahi)
{
    uint64_t r = lo + alo;
    hi += ahi + (r < lo ? 1ull : 0ull);
    lo = r;
}

// Warp, then CTA, then device reduction of a 128-bit sum and the bad flag
// into the state accumulators.  Integer sums: independent of order.
// Must be called by every thread of the CTA; `red` holds 3 * (warps) words.
__device__ __forceinline__ void wl_cta_reduce_to_state(uint64_t lo, uint64_t hi, uint32_t bad,
                                                       WlDevState *st, uint64_t *red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        uint64_t olo = __shfl_down_sync(0xffffffffu, lo, off);
        uint64_t ohi = __shfl_down_sync(0xffffffffu, hi, off);
        wl_add128(lo, hi, olo, ohi);
    }
    bad = __any_sync(0xffffffffu, bad) ? 1u : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        red[warp] = lo;
        red[nw + warp] = hi;
        red[2 * nw + warp] = bad;
    }
    __syncthreads();
    if (warp == 0) {
        lo = lane < nw ? red[lane] : 0ull;
        hi = lane < nw ? red[nw + lane] : 0ull;
        bad = lane < nw ? (uint32_t)red[2 * nw + lane] : 0u;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            uint64_t olo = __shfl_down_sync(0xffffffffu, lo, off);
            uint64_t ohi = __shfl_down_sync(0xffffffffu, hi, off);
            wl_add128(lo, hi, olo, ohi);
        }
        bad = __any_sync(0xffffffffu, bad) ? 1u : 0u;
        if (lane == 0) {
            // fire-and-forget adds: each limb sum stays below 2^64 for up to
            // 2^32 CTAs, so no carry has to travel between the limbs here
            atomicAdd((unsigned long long *)&st->acc0, (unsigned long long)(lo & 0xffffffffull));
            atomicAdd((unsigned long long *)&st->acc1, (unsigned long long)(lo >> 32));
            if (hi)
                atomicAdd((unsigned long long *)&st->acc2, (unsigned long long)hi);
            if (bad)
                atomicOr(&st->acc_bad, 1u);
        }
    }
}

// The pass's Q = acc0 + acc1 2^32 + acc2 2^64 as a 128-bit integer.
__device__ __forceinline__ void wl_acc_read(WlDevState *st, uint64_t &lo, uint64_t &hi)
{
    volatile WlDevState *vs = st;
    const uint64_t a0 = vs->acc0, a1 = vs->acc1, a2 = vs->acc2;
    const uint64_t t = a0 + (a1 << 32);
    hi = a2 + (a1 >> 32) + (t < a0 ? 1ull : 0ull);
    lo = t;
}

// The draws of one pass into a strides slot: 2n uniforms for the strides
// and offsets, then (per-pass sign patterns on) one whose top n bits are
// the pattern (Section 3 prefers a different orthogonal matrix each pass).
//
// RANN4's rotation (n = 2, Section 8): one more uniform U; its top bit is the
// sign of theta, the next bit the range (pi/6..pi/3 or 2pi/3..5pi/6), and the
// low 30 bits place t = tan(theta/2) uniformly in [2 - sqrt 3, 1/sqrt 3] or
// [sqrt 3, 2 + sqrt 3]; cos = (1 - t^2)/(1 + t^2), sin = 2t/(1 + t^2).
__device__ inline void wl_draw_rotation(uint64_t &s, double &cs, double &sn)
{
    const uint32_t u = wl_lcg_step(s);
    const double r3 = __dsqrt_rn(3.0);
    double lo, hi;
    if (((u >> 30) & 1u) == 0) {
        lo = __dsub_rn(2.0, r3);
        hi = __ddiv_rn(r3, 3.0);
    } else {
        lo = r3;
        hi = __dadd_rn(2.0, r3);
    }
    const double f = __dmul_rn((double)(u & 0x3FFFFFFFu), 1.0 / 1073741824.0);
    double t = __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), f));
    if (u >> 31)
        t = -t;
    const double t2 = __dmul_rn(t, t);
    const double den = __dadd_rn(1.0, t2);
    cs = __ddiv_rn(__dsub_rn(1.0, t2), den);
    sn = __ddiv_rn(__dadd_rn(t, t), den);
}

__device__ __forceinline__ void wl_draw_pass(int n, int64_t N, uint64_t &s, WlStrides &slot,
                                             int msigns, const int32_t *ctab)
{
    wl_draw_params(n, N, s, slot.alpha, slot.gamma, ctab);
    slot.signs = msigns ? wl_lcg_step(s) >> (32 - n) : 0u;
    if (n == 2)
        wl_draw_rotation(s, slot.rcos, slot.rsin);
}

// Negate g when bit i of the pattern is set (a sign-bit flip: exact).
__device__ __forceinline__ float wl_sgn(float g, uint32_t signs, int i)
{
    return __uint_as_float(__float_as_uint(g) ^ (((signs >> i) & 1u) << 31));
}
__device__ __forceinline__ double wl_sgn(double g, uint32_t signs, int i)
{
    return __longlong_as_double(__double_as_longlong(g) ^ ((long long)((signs >> i) & 1u) << 63));
}

// With k = st->passes (already counted): `next` takes pass k's strides from
// their slot and pass k + 1's are drawn into the other.  s is the uniform
// state after the draw for pass k, rep the state before it.
__device__ inline void wl_advance_strides(WlDevState *st, int n, int64_t N, uint64_t s, uint64_t rep,
                                          int msigns)
{
    const int64_t k = st->passes;
    const WlStrides &cur = st->ahead[k & 1];
    for (int i = 0; i < 8; i++) {
        st->next.alpha[i] = cur.alpha[i];
        st->next.gamma[i] = cur.gamma[i];
    }
    st->next.signs = cur.signs;
    st->next.rcos = cur.rcos;
    st->next.rsin = cur.rsin;
    st->lcg_rep = rep;
    st->lcg_pend = s;
    wl_draw_pass(n, N, s, st->ahead[(k + 1) & 1], msigns, st->cand);
    st->lcg = s;
}

// ---- end of pass: chi-squared rescale (Eq. 3) and drift monitor ------------
// The chi-squared sample S from the withheld value x (Section 4).  chi = 0:
// Eq. 3, S = (x + sqrt(2 nu - 1))^2 / 2.  chi = 1: Wilson and Hilferty's cube
// (Abramowitz and Stegun 26.4.17), a = 2/(9 nu), S = nu (1 - a + x sqrt(a))^3,
// one of the more accurate approximations the section points to; a sample
// that is not positive marks the pool corrupt (c stays 1).
__device__ __forceinline__ double wl_chi_sample(int chi, int64_t nu, double x)
{
    const double dnu = (double)nu;
    if (!chi) {
        const double r = __dsqrt_rn(__dsub_rn(__dmul_rn(2.0, dnu), 1.0));
        const double xr = __dadd_rn(x, r);
        return __dmul_rn(__dmul_rn(xr, xr), 0.5);
    }
    const double a = __ddiv_rn(2.0, __dmul_rn(9.0, dnu));
    const double b = __dsqrt_rn(a);
    const double t = __dadd_rn(__dsub_rn(1.0, a), __dmul_rn(x, b));
    return __dmul_rn(__dmul_rn(__dmul_rn(t, t), t), dnu);
}

// One thread.  x is the withheld last value of the new pool; with
// r = sqrt(2 nu - 1), S = (x + r)^2 / 2; the next pass scales A by
// c = sqrt(S / q).  q / S_prev - 1 beyond 1e-3 means the pool was overwritten
// (Section 8).  Then the next pass's parameters are drawn.
// kind: what made the pool -- WL_FIN_INIT (creation: the strides of the
// first two passes are drawn), WL_FIN_PASS (a pass: the strides advance),
// WL_FIN_RESTART (a Box-Muller refill, Section 5: the drift history restarts,
// the strides and the pass count are untouched), or WL_FIN_SCALE (a pass whose
// caller holds the parameters: only Q, S and the next scale c are computed --
// no drift check, no stride draw).
#define WL_FIN_INIT 0
#define WL_FIN_PASS 1
#define WL_FIN_RESTART 2
#define WL_FIN_SCALE 3
// local: st is a CTA's shared-memory copy of the state (a run of many passes
// on one CTA), so no device-scope fence is needed; rnu > 0: sqrt(2 nu - 1)
// precomputed by the caller (Eq. 3's sample).
__device__ inline void wl_finalise(WlDevState *st, int n, int64_t N, int64_t nu, double x,
                                   bool fp64, int kind, bool local = false, double rnu = 0.0)
{
    volatile WlDevState *vs = st;
    if (local)
        __threadfence_block();
    else
        __threadfence();
    uint64_t lo, hi;
    wl_acc_read(st, lo, hi);
    uint32_t bad = vs->acc_bad;
    double q;
    if (!fp64) {
        q = __dmul_rn(__ull2double_rn(lo), 1.0 / 4294967296.0);
        if (hi != 0)
            bad = 1;
    } else {
        q = __dadd_rn(__ull2double_rn(hi), __dmul_rn(__ull2double_rn(lo), 1.0 / 18446744073709551616.0));
    }
    double S;
    if (rnu > 0.0 && !st->chi) {
        const double xr = __dadd_rn(x, rnu);
        S = __dmul_rn(__dmul_rn(xr, xr), 0.5);
    } else {
        S = wl_chi_sample(st->chi, nu, x);
    }
    double c = 1.0;
    int32_t status = st->status;
    if (bad || (st->chi && !(S > 0.0)) || !(q > 0.0))
        status |= WL_ECORRUPT;
    else
        c = __dsqrt_rn(__ddiv_rn(S, q));
    const bool params = kind == WL_FIN_INIT || kind == WL_FIN_PASS;
    double drift = 0.0;
    if (st->have_prev && params) {
        drift = __dsub_rn(__ddiv_rn(q, st->S_prev), 1.0);
        if (!(fabs(drift) <= 1e-3))
            status |= WL_ECORRUPT;
    }
    st->S_prev = S;
    st->have_prev = 1;
    st->q_lo = lo;
    st->q_hi = hi;
    st->q = q;
    st->S = S;
    st->c = c;
    st->drift = drift;
    st->bad = (int32_t)bad;
    st->status = status;
    if (params) {
        uint64_t s = st->lcg, rep = st->lcg_pend;
        if (kind == WL_FIN_PASS) {
            st->last = st->next;
            st->passes += 1;
        } else {
            // initial pool: fix the stride candidates for this N, and draw
            // the strides of the first pass as well
            if (n != 2)
                st->ncand = wl_stride_candidates(n, N, st->cand);
            rep = s;
            wl_draw_pass(n, N, s, st->ahead[st->passes & 1], st->msigns, st->cand);
        }
        wl_advance_strides(st, n, N, s, rep, st->msigns);
    }
    st->next.c64 = c;
    st->next.c32 = __double2float_rn(c);
    if (n == 2) {
        // the scale folded into the next pass's rotation
        st->next.rc64 = __dmul_rn(c, st->next.rcos);
        st->next.rs64 = __dmul_rn(c, st->next.rsin);
        st->next.rc32 = __double2float_rn(st->next.rc64);
        st->next.rs32 = __double2float_rn(st->next.rs64);
    }
    st->acc0 = 0;
    st->acc1 = 0;
    st->acc2 = 0;
    st->acc_bad = 0;
    __threadfence();
    st->tile_ctr = 0;
    st->ticket = 0;
}

// The same end-of-pass update as wl_finalise (a pass), run by the whole CTA:
// its three independent chains go to three warps -- the scale (S and c,
// Eq. 3), the drift ratio (Section 8) and the next pass's strides -- so their
// binary64 divisions and square roots and the stride draw overlap.  xf()
// returns the withheld last value of the new pool; rnu = sqrt(2 nu - 1),
// correctly rounded (0: computed here); msigns: the generator draws sign
// patterns.  Every thread of the CTA calls.  st may be the device state
// (after the last-CTA ticket, whose acquire and CTA barrier order every
// other CTA's writes before these reads) or a CTA's shared-memory copy.
template <typename XF>
__device__ inline void wl_finalise_par(WlDevState *st, int n, int64_t N, int64_t nu, double rnu, XF xf,
                                       int msigns, bool fp64)
{
    __shared__ double s_S, s_c;
    __shared__ int32_t s_flag[2];
    volatile WlDevState *vs = st;
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0 && warp < 3) {
        if (warp < 2) {
            uint64_t lo, hi;
            wl_acc_read(st, lo, hi);
            const double q = fp64 ? __dadd_rn(__ull2double_rn(hi),
                                              __dmul_rn(__ull2double_rn(lo), 1.0 / 18446744073709551616.0))
                                  : __dmul_rn(__ull2double_rn(lo), 1.0 / 4294967296.0);
            if (warp == 0) {
                const uint32_t bad = (vs->acc_bad != 0u || (!fp64 && hi != 0)) ? 1u : 0u;
                const int chi = vs->chi;
                const double x = xf();
                double S;
                if (!chi && rnu > 0.0) {
                    const double xr = __dadd_rn(x, rnu);
                    S = __dmul_rn(__dmul_rn(xr, xr), 0.5);
                } else {
                    S = wl_chi_sample(chi, nu, x);
                }
                double c = 1.0;
                int32_t f = 0;
                if (bad || (chi && !(S > 0.0)) || !(q > 0.0))
                    f = WL_ECORRUPT;
                else
                    c = __dsqrt_rn(__ddiv_rn(S, q));
                st->q_lo = lo;
                st->q_hi = hi;
                st->q = q;
                st->S = S;
                st->c = c;
                st->bad = (int32_t)bad;
                s_S = S;
                s_c = c;
                s_flag[0] = f;
            } else {
                double drift = 0.0;
                int32_t f = 0;
                if (vs->have_prev) {
                    drift = __dsub_rn(__ddiv_rn(q, vs->S_prev), 1.0);
                    if (!(fabs(drift) <= 1e-3))
                        f = WL_ECORRUPT;
                }
                st->drift = drift;
                s_flag[1] = f;
            }
        } else {
            st->last = st->next;
            st->passes = vs->passes + 1;
            wl_advance_strides(st, n, N, vs->lcg, vs->lcg_pend, msigns);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->next.c64 = s_c;
        st->next.c32 = __double2float_rn(s_c);
        if (n == 2) {
            // the scale folded into the next pass's rotation
            st->next.rc64 = __dmul_rn(s_c, st->next.rcos);
            st->next.rs64 = __dmul_rn(s_c, st->next.rsin);
            st->next.rc32 = __double2float_rn(st->next.rc64);
            st->next.rs32 = __double2float_rn(st->next.rs64);
        }
        st->S_prev = s_S;
        st->have_prev = 1;
        st->status = vs->status | s_flag[0] | s_flag[1];
        // the next pass (another grid, or this CTA after a barrier) reads these
        st->acc0 = 0;
        st->acc1 = 0;
        st->acc2 = 0;
        st->acc_bad = 0;
        st->tile_ctr = 0;
        st->ticket = 0;
    }
}

// One of the three independent chains of a pass's end, run by one thread
// each, on a state no other thread writes meanwhile:
//   role 0 -- the scale: q from the pass's exact sum of squares (lo, hi, bad
//             totals), S from the withheld value x (Eq. 3, or the Wilson-
//             Hilferty sample), c = sqrt(S / q), and the next pass's c32;
//   role 1 -- the pass count and the strides: `next` takes the next pass's
//             strides and the pass after it draws its own;
//   role 2 -- the drift q / S_prev - 1 (Section 8), then S_prev = S.
// Roles 0 and 2 write disjoint fields and add corruption flags atomically.
// The caller copies st->last = st->next at the start of the pass (nothing
// writes `next` during it); for n = 2 the rotation with the scale folded in
// is left to wl_fold_rotation after the three.
__device__ inline void wl_end_pass_role(WlDevState *st, int n, int64_t N, int64_t nu, double rnu, uint64_t lo,
                                        uint64_t hi, uint32_t bad, double x, int role, int msigns, bool fp64)
{
    if (role == 1) {
        st->passes += 1;
        wl_advance_strides(st, n, N, st->lcg, st->lcg_pend, msigns);
        return;
    }
    if (!fp64 && hi != 0)
        bad = 1u;
    const double q = fp64 ? __dadd_rn(__ull2double_rn(hi),
                                      __dmul_rn(__ull2double_rn(lo), 1.0 / 18446744073709551616.0))
                          : __dmul_rn(__ull2double_rn(lo), 1.0 / 4294967296.0);
    const int chi = st->chi;
    double S;
    if (!chi && rnu > 0.0) {
        const double xr = __dadd_rn(x, rnu);
        S = __dmul_rn(__dmul_rn(xr, xr), 0.5);
    } else {
        S = wl_chi_sample(chi, nu, x);
    }
    int32_t f = 0;
    if (role == 0) {
        double c = 1.0;
        if (bad || (chi && !(S > 0.0)) || !(q > 0.0))
            f = WL_ECORRUPT;
        else
            c = __dsqrt_rn(__ddiv_rn(S, q));
        st->q_lo = lo;
        st->q_hi = hi;
        st->q = q;
        st->S = S;
        st->c = c;
        st->bad = (int32_t)bad;
        st->next.c64 = c;
        st->next.c32 = __double2float_rn(c);
    } else {
        double drift = 0.0;
        if (st->have_prev) {
            drift = __dsub_rn(__ddiv_rn(q, st->S_prev), 1.0);
            if (!(fabs(drift) <= 1e-3))
                f = WL_ECORRUPT;
        }
        st->drift = drift;
        st->S_prev = S;
        st->have_prev = 1;
    }
    if (f)
        atomicOr(&st->status, f);
}

// End of a pass that one CTA ran over the whole pool (the CTA's sum is Q):
// the same update as wl_finalise_par with two barriers.  Per-warp partial
// sums go to `red` (3 words per warp); warps 0 and 2 each complete Q and S
// and run the scale (c, Eq. 3) and the drift ratio (Section 8) respectively,
// while warp 1 draws the strides of the pass after next (at least 3 warps).  The caller copies
// st->last = st->next at the start of the pass (nothing writes `next`
// during it), so the two warps write disjoint fields; for n = 2 the
// rotation with the scale folded in (next.rc*, next.rs*) is left to
// wl_fold_rotation, after the barrier.  st: the CTA's shared-memory copy
// of the state.  Every thread calls.
template <typename XF>
__device__ inline void wl_end_pass_cta(WlDevState *st, int n, int64_t N, int64_t nu, double rnu, uint64_t lo,
                                       uint64_t hi, uint32_t bad, uint64_t *red, XF xf, int msigns, bool fp64)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        uint64_t olo = __shfl_down_sync(0xffffffffu, lo, off);
        uint64_t ohi = __shfl_down_sync(0xffffffffu, hi, off);
        wl_add128(lo, hi, olo, ohi);
    }
    bad = __any_sync(0xffffffffu, bad) ? 1u : 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        red[warp] = lo;
        red[nw + warp] = hi;
        red[2 * nw + warp] = bad;
    }
    __syncthreads();
    if (warp == 0 || warp == 2) {
        // both complete Q (and S): warp 0 for the scale, warp 2 for the drift
        lo = lane < nw ? red[lane] : 0ull;
        hi = lane < nw ? red[nw + lane] : 0ull;
        bad = lane < nw ? (uint32_t)red[2 * nw + lane] : 0u;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            uint64_t olo = __shfl_down_sync(0xffffffffu, lo, off);
            uint64_t ohi = __shfl_down_sync(0xffffffffu, hi, off);
            wl_add128(lo, hi, olo, ohi);
        }
        bad = __any_sync(0xffffffffu, bad) ? 1u : 0u;
        if (lane == 0)
            wl_end_pass_role(st, n, N, nu, rnu, lo, hi, bad, xf(), warp, msigns, fp64);
    } else if (warp == 1 && lane == 0) {
        wl_end_pass_role(st, n, N, nu, rnu, 0, 0, 0, 0.0, 1, msigns, fp64);
    }
    __syncthreads();
}

// n = 2: the scale folded into the next pass's rotation (one thread).
__device__ __forceinline__ void wl_fold_rotation(WlDevState *st)
{
    st->next.rc64 = __dmul_rn(st->next.c64, st->next.rcos);
    st->next.rs64 = __dmul_rn(st->next.c64, st->next.rsin);
    st->next.rc32 = __double2float_rn(st->next.rc64);
    st->next.rs32 = __double2float_rn(st->next.rs64);
}

// The grid-wide bulk-copy pass's form: binary32 pool, x read from the new
// pool in device memory.
__device__ inline void wl_finalise_cta(WlDevState *st, int n, int64_t N, int64_t nu, double rnu,
                                       const float *xp, int msigns)
{
    wl_finalise_par(st, n, N, nu, rnu, [xp]() { return (double)__ldcg(xp); }, msigns, false);
}

// A generator's state kept in shared memory while one CTA runs its passes:
// the finaliser's reads and writes and the sum-of-squares atomics stay on
// chip.  Every thread of the CTA calls both; nothing else touches the
// device copy meanwhile.
__device__ inline void wl_state_load(WlDevState *sh, const WlDevState *g)
{
    const uint32_t *src = (const uint32_t *)g;
    uint32_t *dst = (uint32_t *)sh;
    for (int w = threadIdx.x; w < (int)(sizeof(WlDevState) / 4); w += blockDim.x)
        dst[w] = src[w];
    __syncthreads();
}

__device__ inline void wl_state_store(WlDevState *g, const WlDevState *sh)
{
    __syncthreads();
    const uint32_t *src = (const uint32_t *)sh;
    uint32_t *dst = (uint32_t *)g;
    for (int w = threadIdx.x; w < (int)(sizeof(WlDevState) / 4); w += blockDim.x)
        dst[w] = src[w];
}

// sqrt(2 nu - 1) of Eq. 3, as the finaliser would compute it
__device__ __forceinline__ double wl_rnu(int64_t nu)
{
    return __dsqrt_rn(__dsub_rn(__dmul_rn(2.0, (double)nu), 1.0));
}

// Last-CTA detection: after a CTA barrier one thread takes a ticket with an
// acquire-release atomic, which publishes the CTA's writes (release is
// cumulative over the barrier) and, for the CTA that draws the last ticket,
// makes every other CTA's writes visible before the finaliser runs.
__device__ __forceinline__ bool wl_last_cta(WlDevState *st)
{
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;\n"
                     : "=r"(t)
                     : "l"(&st->ticket)
                     : "memory");
        s_last = (t == gridDim.x * gridDim.y * gridDim.z - 1);
    }
    __syncthreads();
    return s_last;
}

// physical offset of logical pool index q (sub-vector-major, row pitch Np);
// pools hold at most 2^30 values, so the division is a 32-bit one
__device__ __forceinline__ int64_t wl_phys(int64_t q, int64_t N, int64_t Np)
{
    const uint32_t i = (uint32_t)q / (uint32_t)N;
    return (int64_t)i * Np + (q - (int64_t)i * N);
}

// physical offset of the pool's last value (the value Eq. 3 withholds)
__device__ __forceinline__ int64_t wl_last_phys(int n, int64_t N, int64_t Np)
{
    return (int64_t)(n - 1) * Np + (N - 1);
}
