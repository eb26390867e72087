// Initial pool of a Wallace generator: Box-Muller pairs from the uniform
// source (Sections 5 and 8 of Brent's RANN4 paper), its exact sum of squares,
// and the first chi-squared target (Eq. 3) -- one launch.
//
// The logarithm and sine/cosine are written here from textbook series in
// binary64 with explicit round-to-nearest operations:
//   ln(w 2^-32): w = 2^e m, m in [sqrt(1/2), sqrt(2)], ln m = 2 atanh(z),
//     z = (m-1)/(m+1), atanh z = sum_{k=0..10} z^(2k+1)/(2k+1), plus
//     (e-32) ln 2 split into a 24-bit head and a tail (Cody and Waite);
//   sin x, cos x on [0, pi/4]: Maclaurin series through x^15 and x^16 in
//     nested form; quadrant and octant reduction of 2 pi u2 are exact because
//     u2 is a multiple of 2^-32.
#include "wl_common.cuh"
#include "wl_launch.h"

namespace {

__device__ __forceinline__ double pow2d(int k) // 2^k for |k| < 1000
{
    return __longlong_as_double((long long)(1023 + k) << 52);
}

__device__ double log_w(uint64_t w)
{
    int e = 63 - __clzll((long long)w);
    double m = __dmul_rn(__ull2double_rn(w), pow2d(-e));
    if (m > 1.4142135623730951) {
        m = __dmul_rn(m, 0.5);
        e = e + 1;
    }
    double z = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    double z2 = __dmul_rn(z, z);
    double p = 1.0 / 21.0;
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 19.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 17.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 15.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 13.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 11.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 9.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 7.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 5.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0 / 3.0);
    p = __dadd_rn(__dmul_rn(p, z2), 1.0);
    double lm = __dmul_rn(2.0, __dmul_rn(z, p));
    double k = (double)(e - 32);
    const double ln2_head = 0.693147182464599609375;
    const double ln2_tail = -1.904654299957768e-09;
    return __dadd_rn(__dmul_rn(k, ln2_head), __dadd_rn(__dmul_rn(k, ln2_tail), lm));
}

// sin and cos of g*pi/2 for 0 <= g <= 1/2
__device__ void sincos_quarter(double g, double &s, double &c)
{
    double x = __dmul_rn(g, 1.5707963267948966);
    double x2 = __dmul_rn(x, x);
    double t = __dsub_rn(1.0, __dmul_rn(x2, 1.0 / 210.0));
    t = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 156.0), t));
    t = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 110.0), t));
    t = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 72.0), t));
    t = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 42.0), t));
    t = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 20.0), t));
    t = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 6.0), t));
    s = __dmul_rn(x, t);
    double u = __dsub_rn(1.0, __dmul_rn(x2, 1.0 / 240.0));
    u = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 182.0), u));
    u = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 132.0), u));
    u = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 90.0), u));
    u = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 56.0), u));
    u = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 30.0), u));
    u = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 1.0 / 12.0), u));
    u = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, 0.5), u));
    c = u;
}

__device__ void box_muller(uint32_t u1, uint32_t u2, float &a, float &b)
{
    double l = log_w((uint64_t)u1 + 1ull);
    double r = __dsqrt_rn(__dmul_rn(-2.0, l));
    uint32_t quad = u2 >> 30;
    uint32_t f = u2 & 0x3FFFFFFFu;
    double sp, cp;
    if (f <= 0x20000000u) {
        sincos_quarter(__dmul_rn((double)f, 1.0 / 1073741824.0), sp, cp);
    } else {
        double sa, ca;
        sincos_quarter(__dmul_rn((double)(0x40000000u - f), 1.0 / 1073741824.0), sa, ca);
        sp = ca;
        cp = sa;
    }
    double cs, sn;
    switch (quad) {
    case 0: cs = cp; sn = sp; break;
    case 1: cs = -sp; sn = cp; break;
    case 2: cs = -cp; sn = -sp; break;
    default: cs = sp; sn = -cp; break;
    }
    a = __double2float_rn(__dmul_rn(r, cs));
    b = __double2float_rn(__dmul_rn(r, sn));
}

template <typename T>
__global__ void __launch_bounds__(256) init_kernel(T *pool, int n, int64_t N, int64_t Np,
                                                   int64_t nu, uint32_t seed, uint32_t stream,
                                                   WlDevState *st)
{
    __shared__ uint64_t red[3 * 8];
    const uint64_t s0 = wl_seed_mix(seed, stream);
    const int64_t npairs = nu / 2;
    const int64_t G = (int64_t)gridDim.x * blockDim.x;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // map for 2G steps, to hop from pair p to pair p + G
    const uint64_t one = wl_lcg_jump(0, 2 * (uint64_t)G);         // C_{2G}
    const uint64_t AG = wl_lcg_jump(1, 2 * (uint64_t)G) - one;     // A_{2G}
    uint64_t s = wl_lcg_jump(s0, 2 * (uint64_t)p);
    uint64_t lo = 0, hi = 0;
    uint32_t bad = 0;
    for (; p < npairs; p += G) {
        uint64_t t = s;
        uint32_t u1 = wl_lcg_step(t);
        uint32_t u2 = wl_lcg_step(t);
        float a, b;
        box_muller(u1, u2, a, b);
        int64_t q = 2 * p;
        pool[wl_phys(q, N, Np)] = (T)a;
        pool[wl_phys(q + 1, N, Np)] = (T)b;
        if (sizeof(T) == 4) {
            wl_add128(lo, hi, wl_term32(a, bad), 0);
            wl_add128(lo, hi, wl_term32(b, bad), 0);
        } else {
            uint64_t tl, th;
            wl_term64((double)a, tl, th, bad);
            wl_add128(lo, hi, tl, th);
            wl_term64((double)b, tl, th, bad);
            wl_add128(lo, hi, tl, th);
        }
        s = AG * s + one;
    }
    wl_cta_reduce_to_state(lo, hi, bad, st, red);
    if (wl_last_cta(st) && threadIdx.x == 0) {
        st->lcg = wl_lcg_jump(s0, (uint64_t)nu);
        double x = (double)__ldcg(&pool[wl_phys(nu - 1, N, Np)]);
        wl_finalise(st, n, N, nu, x, sizeof(T) == 8, false);
    }
}

} // namespace

cudaError_t wl_launch_init(void *pool, int fp64, int n, int64_t N, int64_t Np, uint32_t seed,
                           uint32_t stream_id, WlDevState *st, int sm_count, cudaStream_t stream)
{
    int64_t nu = (int64_t)n * N;
    int64_t npairs = nu / 2;
    int64_t want = (npairs + 255) / 256;
    int64_t cap = (int64_t)sm_count * 8;
    int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    if (fp64)
        init_kernel<double><<<grid, 256, 0, stream>>>((double *)pool, n, N, Np, nu, seed,
                                                      stream_id, st);
    else
        init_kernel<float><<<grid, 256, 0, stream>>>((float *)pool, n, N, Np, nu, seed,
                                                     stream_id, st);
    return cudaGetLastError();
}
