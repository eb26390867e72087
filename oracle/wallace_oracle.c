/*
 * Oracle for Wallace's normal generator, vectorised form (Brent, RANN4).
 *
 * TEST INFRASTRUCTURE ONLY: a plain sequential restatement of the method, used
 * by the tests, the smoke check and the CPU baseline.  It shares nothing with
 * the CUDA library.  Every function names the part of the paper it follows.
 *
 * Arithmetic rules: compiled with -ffp-contract=off and without fast-math, so
 * each +, -, *, / and sqrt below is one IEEE round-to-nearest operation in the
 * written order (binary32 for float, binary64 for double).  Integer work is
 * exact.  Where the paper is silent (the uniform generator, the initial fill,
 * the stride tables, the precision of the sum of squares) this file fixes one
 * reading and says so in place.
 */
#include "wallace_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ *
 * Subsidiary uniform generator (Section 8: RANN4 draws its initial pool and
 * its per-pass parameters from a uniform generator whose recurrence the paper
 * does not print).  Reading fixed here: a 64-bit linear congruential
 * generator s <- a*s + b (mod 2^64) with the multiplier and increment Knuth
 * published for MMIX; each step returns the top 32 bits of the new state.
 * The starting state is SplitMix64 (Steele, Lea and Flood, 2014) applied to
 * (stream << 32 | seed), so that a processor or stream number appended to the
 * seed gives a different sequence (Section 8, DP_VRANU4).
 * ------------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t orc_seed_state(uint32_t seed, uint32_t stream)
{
    return orc_splitmix64(((uint64_t)stream << 32) | (uint64_t)seed);
}

uint32_t orc_lcg_next(uint64_t *state)
{
    *state = *state * 6364136223846793005ULL + 1442695040888963407ULL;
    return (uint32_t)(*state >> 32);
}

/* The state m steps ahead: the step is the affine map s -> a s + b (mod
 * 2^64); m steps compose to s -> A s + B, built by binary powering of the map
 * (F. B. Brown, "Random number generation with arbitrary strides", 1994). */
uint64_t orc_lcg_jump(uint64_t s, uint64_t m)
{
    uint64_t A = 1, B = 0;                          /* accumulated map */
    uint64_t a = 6364136223846793005ULL, b = 1442695040888963407ULL; /* map for 2^k steps */
    while (m) {
        if (m & 1) {
            A = a * A;
            B = a * B + b;
        }
        b = a * b + b;
        a = a * a;
        m >>= 1;
    }
    return A * s + B;
}

/* ------------------------------------------------------------------------ *
 * Elementary functions for the initial Box-Muller fill (Section 5 refills the
 * pool with Box-Muller; Section 8 initialises from the uniform generator).
 * Written from textbook series in binary64 so that the library can reproduce
 * them exactly with the same operations:
 *   ln: w = 2^e * m with m in [sqrt(1/2), sqrt(2)],
 *       ln m = 2 atanh(z), z = (m-1)/(m+1), atanh z = sum z^(2k+1)/(2k+1),
 *       k = 0..10; e*ln 2 is split into a 24-bit head and a tail (Cody-Waite).
 *   sin, cos on [0, pi/4]: Maclaurin series through x^15 and x^16, nested.
 * ------------------------------------------------------------------------ */
static const double ORC_SQRT2 = 1.4142135623730951;
static const double ORC_LN2_HI = 0.693147182464599609375;   /* ln 2 to 24 bits */
static const double ORC_LN2_LO = -1.904654299957768e-09;    /* ln 2 - head     */
static const double ORC_PI_HALF = 1.5707963267948966;

double orc_log_w(uint64_t w)
{
    int e = 0;
    uint64_t t = w;
    while (t >= 2) {
        t >>= 1;
        e++;
    }
    double m = (double)w / (double)((uint64_t)1 << e); /* exact, m in [1,2) */
    if (m > ORC_SQRT2) {
        m = m * 0.5;
        e = e + 1;
    }
    double z = (m - 1.0) / (m + 1.0);
    double z2 = z * z;
    double p = 1.0 / 21.0;
    p = p * z2 + 1.0 / 19.0;
    p = p * z2 + 1.0 / 17.0;
    p = p * z2 + 1.0 / 15.0;
    p = p * z2 + 1.0 / 13.0;
    p = p * z2 + 1.0 / 11.0;
    p = p * z2 + 1.0 / 9.0;
    p = p * z2 + 1.0 / 7.0;
    p = p * z2 + 1.0 / 5.0;
    p = p * z2 + 1.0 / 3.0;
    p = p * z2 + 1.0;
    double lm = 2.0 * (z * p);
    double k = (double)(e - 32);
    return k * ORC_LN2_HI + (k * ORC_LN2_LO + lm);
}

void orc_sincos_quarter(double g, double *s, double *c)
{
    double x = g * ORC_PI_HALF;
    double x2 = x * x;
    /* sin x = x (1 - x^2/(2*3) (1 - x^2/(4*5) (... (1 - x^2/(14*15))))) */
    double t = 1.0 - x2 * (1.0 / 210.0);
    t = 1.0 - (x2 * (1.0 / 156.0)) * t;
    t = 1.0 - (x2 * (1.0 / 110.0)) * t;
    t = 1.0 - (x2 * (1.0 / 72.0)) * t;
    t = 1.0 - (x2 * (1.0 / 42.0)) * t;
    t = 1.0 - (x2 * (1.0 / 20.0)) * t;
    t = 1.0 - (x2 * (1.0 / 6.0)) * t;
    *s = x * t;
    /* cos x = 1 - x^2/(1*2) (1 - x^2/(3*4) (... (1 - x^2/(15*16)))) */
    double u = 1.0 - x2 * (1.0 / 240.0);
    u = 1.0 - (x2 * (1.0 / 182.0)) * u;
    u = 1.0 - (x2 * (1.0 / 132.0)) * u;
    u = 1.0 - (x2 * (1.0 / 90.0)) * u;
    u = 1.0 - (x2 * (1.0 / 56.0)) * u;
    u = 1.0 - (x2 * (1.0 / 30.0)) * u;
    u = 1.0 - (x2 * (1.0 / 12.0)) * u;
    u = 1.0 - (x2 * 0.5) * u;
    *c = u;
}

void orc_sincos_2pi(uint32_t u, double *s, double *c)
{
    /* theta = 2*pi*u/2^32 = q*pi/2 + phi, q = top two bits of u */
    uint32_t q = u >> 30;
    uint32_t f = u & 0x3FFFFFFFu;
    double sp, cp;
    if (f <= 0x20000000u) {
        orc_sincos_quarter((double)f * (1.0 / 1073741824.0), &sp, &cp);
    } else {
        double a, b;
        orc_sincos_quarter((double)(0x40000000u - f) * (1.0 / 1073741824.0), &a, &b);
        sp = b; /* sin(pi/2 - x) = cos x */
        cp = a;
    }
    switch (q) {
    case 0: *c = cp;  *s = sp;  break;
    case 1: *c = -sp; *s = cp;  break;
    case 2: *c = -cp; *s = -sp; break;
    default: *c = sp; *s = -cp; break;
    }
}

/* Box-Muller (Muller 1959, named in Sections 1 and 5): u1 = (U1+1)/2^32 in
 * (0,1], u2 = U2/2^32 in [0,1), r = sqrt(-2 ln u1), theta = 2 pi u2;
 * the pair is (r cos theta, r sin theta), each rounded once to binary32. */
void orc_box_muller(uint32_t u1, uint32_t u2, float *a, float *b)
{
    double l = orc_log_w((uint64_t)u1 + 1u);
    double r = sqrt(-2.0 * l);
    double s, c;
    orc_sincos_2pi(u2, &s, &c);
    *a = (float)(r * c);
    *b = (float)(r * s);
}

/* The Box-Muller method as a generator in its own right: the comparison
 * method of the paper's abstract and Section 1.  Values [offset, offset +
 * count) of the stream of pairs formed from consecutive uniforms of the
 * (seed, stream) source -- the pairs of the initial pool (Sections 5 and 8)
 * -- each mapped to mu + sigma*y (binary32 multiply, then add). */
void orc_boxmuller_stream(uint32_t seed, uint32_t stream, int64_t offset, int64_t count,
                          float mu, float sigma, float *out)
{
    uint64_t s = orc_seed_state(seed, stream);
    int64_t p0 = offset / 2;
    for (int64_t k = 0; k < 2 * p0; k++)
        (void)orc_lcg_next(&s);
    int64_t v = 2 * p0; /* value index of the next pair's first value */
    int64_t done = 0;
    while (done < count) {
        uint32_t u1 = orc_lcg_next(&s);
        uint32_t u2 = orc_lcg_next(&s);
        float y[2];
        orc_box_muller(u1, u2, &y[0], &y[1]);
        for (int h = 0; h < 2; h++, v++) {
            if (v >= offset && done < count) {
                float t = sigma * y[h];
                out[done++] = mu + t;
            }
        }
    }
}

/* ------------------------------------------------------------------------ *
 * Per-pass parameters (Eq. 1 and Eq. 2; Sections 3, 7 and 8).  The paper asks
 * for strides that are distinct, greater than one, odd, and coprime to N, and
 * offsets uniform on {0..N-1}, all redrawn every pass; RANN4 picks its two
 * strides from {3,5} and {7,11}.  Reading for n = 4 and n = 8 (the paper
 * gives only n = 2; this rule is a choice made for the GPU's lane tiling,
 * whose lane count is the strides' lcm, within those constraints -- the
 * paper itself asks nothing of the lcm): with p < q < r the three smallest odd primes that do not
 * divide N, the candidate strides are the odd divisors > 1 of p^2 q (n = 4:
 * five values) or of p^2 q r (n = 8: eleven values), in increasing order.
 * Every candidate is then coprime to N and the lcm of any pass's strides
 * divides p^2 q or p^2 q r; for N coprime to 15 the n = 4 set is
 * {3, 5, 9, 15, 45}, and for N coprime to 105 the n = 8 set is the odd
 * divisors of 315.  Sub-vector i draws one uniform U and takes entry
 * floor(U * k / 2^32) of the k candidates not yet used this pass, in order,
 * so every ordered choice of distinct strides is equally likely (120 for
 * n = 4).  For n = 2 the candidates are RANN4's pair for the sub-vector,
 * those coprime to N; if neither is, it takes the smallest odd number > 1
 * coprime to N and not in use.  Then one uniform U gives the offset
 * floor(U * N / 2^32).
 * ------------------------------------------------------------------------ */
static int64_t orc_gcd(int64_t a, int64_t b)
{
    while (b != 0) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static int orc_stride_ok(int32_t a, int64_t N, const int32_t *used, int nused)
{
    if (orc_gcd(a, N) != 1)
        return 0;
    for (int k = 0; k < nused; k++)
        if (used[k] == a)
            return 0;
    return 1;
}

/* The odd primes below 64.  The product of the first fifteen exceeds 2^63,
 * so at most fourteen of them divide an N < 2^63 and at least three do not. */
static const int32_t ORC_ODD_PRIMES[17] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61};

/* Candidate strides of the reading above for n = 4 or 8, increasing; returns
 * how many (5 or 11). */
int orc_stride_candidates(int n, int64_t N, int32_t *cand)
{
    int32_t pr[3];
    int np = 0;
    const int need = n == 8 ? 3 : 2;
    for (int k = 0; k < 17 && np < need; k++)
        if (N % ORC_ODD_PRIMES[k] != 0)
            pr[np++] = ORC_ODD_PRIMES[k];
    /* odd divisors of p^2 q (r): p^e1 q^e2 r^e3, e1 <= 2, e2 <= 1, e3 <= 1 */
    int nc = 0;
    const int e3max = n == 8 ? 1 : 0;
    for (int e1 = 0; e1 <= 2; e1++)
        for (int e2 = 0; e2 <= 1; e2++)
            for (int e3 = 0; e3 <= e3max; e3++) {
                int32_t d = 1;
                for (int t = 0; t < e1; t++)
                    d *= pr[0];
                if (e2)
                    d *= pr[1];
                if (e3)
                    d *= pr[2];
                if (d > 1)
                    cand[nc++] = d;
            }
    /* insertion sort: increasing order */
    for (int a = 1; a < nc; a++) {
        int32_t v = cand[a];
        int b = a - 1;
        while (b >= 0 && cand[b] > v) {
            cand[b + 1] = cand[b];
            b--;
        }
        cand[b + 1] = v;
    }
    return nc;
}

/* n = 2 is RANN4 itself (Section 8): alpha from {3, 5} for x and beta from
 * {7, 11} for y, each drawn as above among the candidates still available. */
static const int32_t ORC_CAND2[2][2] = {{3, 5}, {7, 11}};

void orc_draw_params(int n, int64_t N, uint64_t *state, int32_t *alpha, int64_t *gamma)
{
    int32_t table[11];
    int ntable = 0;
    if (n != 2)
        ntable = orc_stride_candidates(n, N, table);
    for (int i = 0; i < n; i++) {
        const int32_t *cand = n == 2 ? ORC_CAND2[i] : table;
        const int ncand = n == 2 ? 2 : ntable;
        uint32_t us = orc_lcg_next(state);
        int32_t avail[11];
        int na = 0;
        for (int k = 0; k < ncand; k++)
            if (orc_stride_ok(cand[k], N, alpha, i))
                avail[na++] = cand[k];
        int32_t a;
        if (na > 0) {
            a = avail[((uint64_t)us * (uint64_t)na) >> 32];
        } else {
            a = 3;
            while (!orc_stride_ok(a, N, alpha, i))
                a += 2;
        }
        alpha[i] = a;
        uint32_t uo = orc_lcg_next(state);
        gamma[i] = (int64_t)(((uint64_t)uo * (uint64_t)N) >> 32);
    }
}

/* ------------------------------------------------------------------------ *
 * RANN4's rotation (Section 8, n = 2): A = [[cos t, sin t], [-sin t, cos t]]
 * with pi/6 <= |theta| <= pi/3 or 2 pi/3 <= |theta| <= 5 pi/6, so that
 * min(|sin|, |cos|) >= 1/2; a uniform selects t = tan(theta/2) and
 *     cos theta = (1 - t^2) / (1 + t^2),  sin theta = 2 t / (1 + t^2).
 * Reading (the paper writes |theta| for the first range and theta for the
 * second): both ranges for either sign of theta.  One uniform U per pass,
 * drawn after the strides and offsets: its top two bits pick the range --
 * t in [2 - sqrt 3, 1/sqrt 3] (theta in [pi/6, pi/3]), [sqrt 3, 2 + sqrt 3]
 * (theta in [2 pi/3, 5 pi/6]), or their negatives -- and its low 30 bits
 * place t uniformly in it: t = lo + (hi - lo) (U mod 2^30) 2^-30.
 * ------------------------------------------------------------------------ */
void orc_draw_rotation(uint64_t *state, double *cs, double *sn)
{
    uint32_t u = orc_lcg_next(state);
    double r3 = sqrt(3.0);
    double lo, hi;
    if (((u >> 30) & 1u) == 0) {
        lo = 2.0 - r3;
        hi = r3 / 3.0;
    } else {
        lo = r3;
        hi = 2.0 + r3;
    }
    double f = (double)(u & 0x3FFFFFFFu) * (1.0 / 1073741824.0);
    double t = lo + (hi - lo) * f;
    if (u >> 31)
        t = -t;
    double t2 = t * t;
    double den = 1.0 + t2;
    *cs = (1.0 - t2) / den;
    *sn = (t + t) / den;
}

/* One RANN4 pass (Eq. 1 with n = 2): x'_j = C g0 + S g1, y'_j = C g1 - S g0,
 * g0 = x[(alpha j + gamma) mod N], g1 = y[(beta j + delta) mod N], where the
 * chi-squared scale is folded into the rotation: C = c cos theta and
 * S = c sin theta, rounded once to the pool's precision. */
void orc_pass_rot32(int64_t N, const float *x, float *y, const int32_t *alpha,
                    const int64_t *gamma, float C, float S)
{
    for (int64_t j = 0; j < N; j++) {
        uint64_t i0 = ((uint64_t)alpha[0] * (uint64_t)j + (uint64_t)gamma[0]) % (uint64_t)N;
        uint64_t i1 = ((uint64_t)alpha[1] * (uint64_t)j + (uint64_t)gamma[1]) % (uint64_t)N;
        float g0 = x[(int64_t)i0], g1 = x[N + (int64_t)i1];
        float a = C * g0, b = S * g1;
        float d = C * g1, e = S * g0;
        y[j] = a + b;
        y[N + j] = d - e;
    }
}

void orc_pass_rot64(int64_t N, const double *x, double *y, const int32_t *alpha,
                    const int64_t *gamma, double C, double S)
{
    for (int64_t j = 0; j < N; j++) {
        uint64_t i0 = ((uint64_t)alpha[0] * (uint64_t)j + (uint64_t)gamma[0]) % (uint64_t)N;
        uint64_t i1 = ((uint64_t)alpha[1] * (uint64_t)j + (uint64_t)gamma[1]) % (uint64_t)N;
        double g0 = x[(int64_t)i0], g1 = x[N + (int64_t)i1];
        double a = C * g0, b = S * g1;
        double d = C * g1, e = S * g0;
        y[j] = a + b;
        y[N + j] = d - e;
    }
}

/* ------------------------------------------------------------------------ *
 * The orthogonal transform (Section 2; the n-by-n generalisation stated in
 * Sections 1 and 9).  A = (2/n) J - I (J the all-ones matrix) is orthogonal
 * and symmetric, entries +-1/2 for n = 4 and 1/4, -3/4 for n = 8.  With the
 * chi-squared scale c of Section 4 folded into A:
 *     s = pairwise sum of g,  h = s * (2/n),  y_k = (h - g_k) * c.
 * ------------------------------------------------------------------------ */
void orc_transform32(int n, const float *g, float c, float *y)
{
    float s, h;
    if (n == 4) {
        float a = g[0] + g[1];
        float b = g[2] + g[3];
        s = a + b;
        h = s * 0.5f;
    } else {
        float a = g[0] + g[1];
        float b = g[2] + g[3];
        float d = g[4] + g[5];
        float e = g[6] + g[7];
        float ab = a + b;
        float de = d + e;
        s = ab + de;
        h = s * 0.25f;
    }
    for (int k = 0; k < n; k++) {
        float t = h - g[k];
        y[k] = t * c;
    }
}

void orc_transform64(int n, const double *g, double c, double *y)
{
    double s, h;
    if (n == 4) {
        double a = g[0] + g[1];
        double b = g[2] + g[3];
        s = a + b;
        h = s * 0.5;
    } else {
        double a = g[0] + g[1];
        double b = g[2] + g[3];
        double d = g[4] + g[5];
        double e = g[6] + g[7];
        double ab = a + b;
        double de = d + e;
        s = ab + de;
        h = s * 0.25;
    }
    for (int k = 0; k < n; k++) {
        double t = h - g[k];
        y[k] = t * c;
    }
}

/* One pass, Eq. 1 with n sub-vectors: x'_i[j] = (A D g)_i, g_i = x_i[(alpha_i j +
 * gamma_i) mod N], j = 0..N-1, into a second buffer (double buffering,
 * Section 2).  Pool layout: sub-vector i occupies x[i*N .. i*N+N-1].
 * D = diag(+-1): bit i of `signs` negates g_i (0 for the fixed matrix A;
 * Section 3 prefers a different orthogonal matrix at each pass, and A D is
 * orthogonal for every sign pattern). */
void orc_pass_explicit32(int n, int64_t N, const float *x, float *y,
                         const int32_t *alpha, const int64_t *gamma, float c, uint32_t signs)
{
    float g[8], t[8];
    for (int64_t j = 0; j < N; j++) {
        for (int i = 0; i < n; i++) {
            uint64_t idx = ((uint64_t)alpha[i] * (uint64_t)j + (uint64_t)gamma[i]) % (uint64_t)N;
            g[i] = x[(int64_t)i * N + (int64_t)idx];
            if ((signs >> i) & 1u)
                g[i] = -g[i];
        }
        orc_transform32(n, g, c, t);
        for (int k = 0; k < n; k++)
            y[(int64_t)k * N + j] = t[k];
    }
}

void orc_pass_explicit64(int n, int64_t N, const double *x, double *y,
                         const int32_t *alpha, const int64_t *gamma, double c, uint32_t signs)
{
    double g[8], t[8];
    for (int64_t j = 0; j < N; j++) {
        for (int i = 0; i < n; i++) {
            uint64_t idx = ((uint64_t)alpha[i] * (uint64_t)j + (uint64_t)gamma[i]) % (uint64_t)N;
            g[i] = x[(int64_t)i * N + (int64_t)idx];
            if ((signs >> i) & 1u)
                g[i] = -g[i];
        }
        orc_transform64(n, g, c, t);
        for (int k = 0; k < n; k++)
            y[(int64_t)k * N + j] = t[k];
    }
}

/* ------------------------------------------------------------------------ *
 * Sum of squares (Section 4, and the drift monitor of Section 8).  Reading:
 * the accumulation must not depend on summation order, so Q is an exact
 * integer.  FP32 pool: Q = sum floor(y^2 * 2^32); y^2 of a binary32 value is
 * exact in binary64 and so is the scaling, hence each term is exact.  FP64
 * pool: Q = sum floor(fl(y*y) * 2^64), fl() one binary64 rounding.  A value
 * that is not finite or has |y| >= 256 cannot come from a sane pool; it
 * contributes nothing and flags the pool as corrupt.
 * ------------------------------------------------------------------------ */
uint64_t orc_term32(float y, int *bad)
{
    double d = (double)y;
    if (!(fabs(d) < 256.0)) {
        *bad = 1;
        return 0;
    }
    return (uint64_t)floor(d * d * 4294967296.0);
}

static unsigned __int128 orc_term64(double y, int *bad)
{
    if (!(fabs(y) < 256.0)) {
        *bad = 1;
        return 0;
    }
    double t = y * y;
    double f = floor(ldexp(t, 64));
    return (unsigned __int128)f;
}

int orc_sumsq32(const float *pool, int64_t nu, uint64_t *q_lo, uint64_t *q_hi)
{
    unsigned __int128 acc = 0;
    int bad = 0;
    for (int64_t q = 0; q < nu; q++)
        acc += orc_term32(pool[q], &bad);
    *q_lo = (uint64_t)acc;
    *q_hi = (uint64_t)(acc >> 64);
    return bad;
}

int orc_sumsq64(const double *pool, int64_t nu, uint64_t *q_lo, uint64_t *q_hi)
{
    unsigned __int128 acc = 0;
    int bad = 0;
    for (int64_t q = 0; q < nu; q++)
        acc += orc_term64(pool[q], &bad);
    *q_lo = (uint64_t)acc;
    *q_hi = (uint64_t)(acc >> 64);
    return bad;
}

/* Section 6: a fraction 1/f of each pool is returned.  Reading: the returned
 * values are the first R = min(floor(frac * nu), nu - 1) entries of the new
 * pool; the last entry is never returned because it feeds Eq. 3. */
int64_t orc_returned_count(int64_t nu, double frac)
{
    double r = floor(frac * (double)nu);
    int64_t R = (int64_t)r;
    if (R > nu - 1)
        R = nu - 1;
    if (R < 0)
        R = 0;
    return R;
}

/* ------------------------------------------------------------------------ *
 * A whole generator.
 * ------------------------------------------------------------------------ */
struct orc_gen {
    int n, mode, chi, msigns;
    uint32_t seed, stream;
    int64_t restart; /* refill interval in passes (0: never) */
    int64_t N, nu, R;
    double frac;
    float *p32[2];
    double *p64[2];
    int cur;
    uint64_t lcg;
    double S_prev;
    int have_prev;
    orc_stats st;
};

/* Section 4 (Eq. 3) and Section 8: after a pool is made, its last value x
 * gives a chi-squared sample S = (x + sqrt(2 nu - 1))^2 / 2; the next pass
 * scales A by c = sqrt(S / q) so that the next pool's sum of squares is S.
 * The ratio q_k / S_{k-1} - 1 is the drift the monitor watches; beyond 1e-3
 * the work area is taken to be overwritten.
 *
 * With ORC_CHI_WH the sample is Wilson and Hilferty's cube instead, one of
 * the more accurate approximations Section 4 points to (Abramowitz and
 * Stegun 26.4.17): with a = 2/(9 nu), S = nu (1 - a + x sqrt(a))^3.  A
 * sample that is not positive (x below -(1 - a)/sqrt(a)) marks the pool
 * corrupt and keeps c = 1, as a non-positive q does. */
static void orc_finalise(orc_gen *g)
{
    uint64_t lo, hi;
    int bad;
    double x, q;
    if (g->mode == ORC_FP32) {
        bad = orc_sumsq32(g->p32[g->cur], g->nu, &lo, &hi);
        x = (double)g->p32[g->cur][g->nu - 1];
        q = (double)lo * (1.0 / 4294967296.0);
        if (hi != 0)
            bad = 1;
    } else {
        bad = orc_sumsq64(g->p64[g->cur], g->nu, &lo, &hi);
        x = g->p64[g->cur][g->nu - 1];
        q = (double)hi + (double)lo * (1.0 / 18446744073709551616.0);
    }
    double S;
    int bad_s = 0;
    if (!g->chi) {
        double r = sqrt(2.0 * (double)g->nu - 1.0);
        double xr = x + r;
        S = (xr * xr) * 0.5;
    } else {
        double a = 2.0 / (9.0 * (double)g->nu);
        double b = sqrt(a);
        double t = (1.0 - a) + x * b;
        S = ((t * t) * t) * (double)g->nu;
        bad_s = !(S > 0.0);
    }
    double c = 1.0;
    if (bad || bad_s || !(q > 0.0)) {
        g->st.status |= ORC_ECORRUPT;
    } else {
        c = sqrt(S / q);
    }
    double drift = 0.0;
    if (g->have_prev) {
        drift = q / g->S_prev - 1.0;
        if (!(fabs(drift) <= 1e-3))
            g->st.status |= ORC_ECORRUPT;
    }
    g->S_prev = S;
    g->have_prev = 1;
    g->st.q_lo = lo;
    g->st.q_hi = hi;
    g->st.q = q;
    g->st.S = S;
    g->st.c = c;
    g->st.c32 = (float)c;
    g->st.drift = drift;
    g->st.bad = bad;
}

orc_gen *orc_create(int n, int64_t N, uint32_t seed, uint32_t stream, double frac, int mode)
{
    if ((n != 2 && n != 4 && n != 8) || N < 4 || (int64_t)n * N > ((int64_t)1 << 30))
        return NULL;
    if (n == 2 && (mode & ORC_SIGNS))
        return NULL; /* RANN4 draws its own rotation each pass */
    int chi = (mode & ORC_CHI_WH) != 0;
    int msigns = (mode & ORC_SIGNS) != 0;
    mode &= ~(ORC_CHI_WH | ORC_SIGNS);
    if (!(frac > 0.0 && frac <= 1.0) || (mode != ORC_FP32 && mode != ORC_FP64))
        return NULL;
    int64_t nu = (int64_t)n * N;
    int64_t R = orc_returned_count(nu, frac);
    if (R < 1)
        return NULL;
    orc_gen *g = (orc_gen *)calloc(1, sizeof(orc_gen));
    if (!g)
        return NULL;
    g->n = n;
    g->chi = chi;
    g->msigns = msigns;
    g->seed = seed;
    g->stream = stream;
    g->N = N;
    g->nu = nu;
    g->R = R;
    g->frac = frac;
    g->mode = mode;
    g->p32[0] = (float *)calloc((size_t)nu, sizeof(float));
    g->p32[1] = (float *)calloc((size_t)nu, sizeof(float));
    if (!g->p32[0] || !g->p32[1]) {
        orc_destroy(g);
        return NULL;
    }
    if (mode == ORC_FP64) {
        g->p64[0] = (double *)calloc((size_t)nu, sizeof(double));
        g->p64[1] = (double *)calloc((size_t)nu, sizeof(double));
        if (!g->p64[0] || !g->p64[1]) {
            orc_destroy(g);
            return NULL;
        }
    }
    g->lcg = orc_seed_state(seed, stream);
    /* initial pool: Box-Muller pairs from consecutive uniforms */
    for (int64_t p = 0; p < nu / 2; p++) {
        uint32_t u1 = orc_lcg_next(&g->lcg);
        uint32_t u2 = orc_lcg_next(&g->lcg);
        orc_box_muller(u1, u2, &g->p32[0][2 * p], &g->p32[0][2 * p + 1]);
    }
    if (mode == ORC_FP64)
        for (int64_t q = 0; q < nu; q++)
            g->p64[0][q] = (double)g->p32[0][q];
    g->cur = 0;
    orc_finalise(g);
    g->st.passes = 0;
    g->st.R = R;
    g->st.cursor = R; /* the initial pool is not returned */
    g->st.lcg = g->lcg;
    return g;
}

/* Section 5 (Restarting): the pool is refilled by Box-Muller from the
 * uniform source and the chi-squared sample, scale and drift history are
 * taken afresh from it, as at creation.  Reading: restart r = 1, 2, ... takes
 * the uniforms at positions [r 2^40, r 2^40 + nu) of the generator's LCG
 * sequence (its seed state jumped r 2^40 steps): apart from the initial pool
 * (positions [0, nu)) and the per-pass draws (2n a pass from position nu), so
 * no uniform serves twice, and the draws of later passes are unchanged.  The
 * refilled pool is not returned. */
void orc_restart_pool(uint32_t seed, uint32_t stream, int64_t r, int64_t nu, float *pool)
{
    uint64_t s = orc_lcg_jump(orc_seed_state(seed, stream), (uint64_t)r << 40);
    for (int64_t q = 0; q < nu / 2; q++) {
        uint32_t u1 = orc_lcg_next(&s);
        uint32_t u2 = orc_lcg_next(&s);
        orc_box_muller(u1, u2, &pool[2 * q], &pool[2 * q + 1]);
    }
}

static void orc_restart(orc_gen *g, int64_t r)
{
    float *p = g->p32[g->cur];
    orc_restart_pool(g->seed, g->stream, r, g->nu, p);
    if (g->mode == ORC_FP64)
        for (int64_t q = 0; q < g->nu; q++)
            g->p64[g->cur][q] = (double)p[q];
    g->have_prev = 0;
    orc_finalise(g);
}

void orc_set_restart(orc_gen *g, int64_t interval)
{
    g->restart = interval > 0 ? interval : 0;
}

int orc_pass(orc_gen *g)
{
    /* after every `restart` passes, refill before the next pass */
    if (g->restart > 0 && g->st.passes > 0 && g->st.passes % g->restart == 0)
        orc_restart(g, g->st.passes / g->restart);
    orc_draw_params(g->n, g->N, &g->lcg, g->st.alpha, g->st.gamma);
    /* ORC_SIGNS (reading of Section 3's per-pass matrices): one more uniform
     * per pass; its top n bits are the sign pattern of D_k */
    g->st.signs = g->msigns ? orc_lcg_next(&g->lcg) >> (32 - g->n) : 0u;
    int src = g->cur, dst = 1 - g->cur;
    if (g->n == 2) {
        orc_draw_rotation(&g->lcg, &g->st.rot_c, &g->st.rot_s);
        if (g->mode == ORC_FP32)
            orc_pass_rot32(g->N, g->p32[src], g->p32[dst], g->st.alpha, g->st.gamma,
                           (float)(g->st.c * g->st.rot_c), (float)(g->st.c * g->st.rot_s));
        else
            orc_pass_rot64(g->N, g->p64[src], g->p64[dst], g->st.alpha, g->st.gamma,
                           g->st.c * g->st.rot_c, g->st.c * g->st.rot_s);
    } else if (g->mode == ORC_FP32)
        orc_pass_explicit32(g->n, g->N, g->p32[src], g->p32[dst], g->st.alpha, g->st.gamma,
                            g->st.c32, g->st.signs);
    else
        orc_pass_explicit64(g->n, g->N, g->p64[src], g->p64[dst], g->st.alpha, g->st.gamma,
                            g->st.c, g->st.signs);
    g->cur = dst;
    g->st.passes++;
    orc_finalise(g);
    g->st.cursor = 0;
    g->st.lcg = g->lcg;
    return g->st.status;
}

/* The user call of Section 8: any count, any mu and sigma per call; the
 * stream of returned values does not depend on how it is split into calls. */
int orc_fill32(orc_gen *g, float *out, int64_t count, float mu, float sigma)
{
    if (g->mode != ORC_FP32 || count < 0)
        return ORC_EINVAL;
    int64_t done = 0;
    while (done < count) {
        if (g->st.cursor >= g->R)
            orc_pass(g);
        int64_t take = g->R - g->st.cursor;
        if (take > count - done)
            take = count - done;
        const float *pool = g->p32[g->cur];
        for (int64_t k = 0; k < take; k++) {
            float t = sigma * pool[g->st.cursor + k];
            out[done + k] = mu + t;
        }
        g->st.cursor += take;
        done += take;
    }
    return g->st.status;
}

int orc_fill64(orc_gen *g, double *out, int64_t count, double mu, double sigma)
{
    if (g->mode != ORC_FP64 || count < 0)
        return ORC_EINVAL;
    int64_t done = 0;
    while (done < count) {
        if (g->st.cursor >= g->R)
            orc_pass(g);
        int64_t take = g->R - g->st.cursor;
        if (take > count - done)
            take = count - done;
        const double *pool = g->p64[g->cur];
        for (int64_t k = 0; k < take; k++) {
            double t = sigma * pool[g->st.cursor + k];
            out[done + k] = mu + t;
        }
        g->st.cursor += take;
        done += take;
    }
    return g->st.status;
}

void orc_get_pool32(const orc_gen *g, float *out)
{
    if (g->mode == ORC_FP32)
        memcpy(out, g->p32[g->cur], (size_t)g->nu * sizeof(float));
    else
        for (int64_t q = 0; q < g->nu; q++)
            out[q] = (float)g->p64[g->cur][q];
}

void orc_get_pool64(const orc_gen *g, double *out)
{
    if (g->mode == ORC_FP64)
        memcpy(out, g->p64[g->cur], (size_t)g->nu * sizeof(double));
    else
        for (int64_t q = 0; q < g->nu; q++)
            out[q] = (double)g->p32[g->cur][q];
}

void orc_set_pool32(orc_gen *g, const float *pool)
{
    memcpy(g->p32[g->cur], pool, (size_t)g->nu * sizeof(float));
    if (g->mode == ORC_FP64)
        for (int64_t q = 0; q < g->nu; q++)
            g->p64[g->cur][q] = (double)pool[q];
}

void orc_get_stats(const orc_gen *g, orc_stats *st)
{
    *st = g->st;
}

void orc_destroy(orc_gen *g)
{
    if (!g)
        return;
    free(g->p32[0]);
    free(g->p32[1]);
    free(g->p64[0]);
    free(g->p64[1]);
    free(g);
}
