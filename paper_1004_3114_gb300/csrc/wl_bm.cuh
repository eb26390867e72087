// Box-Muller pairs from two 32-bit uniforms in binary64 with explicit
// round-to-nearest operations (Sections 5 and 8 of Brent's RANN4 paper: the
// initial pool, and the comparison method of the paper's introduction):
//   u1 = (U1 + 1) 2^-32 in (0, 1], u2 = U2 2^-32 in [0, 1);
//   r = sqrt(-2 ln u1), (a, b) = (r cos 2 pi u2, r sin 2 pi u2).
// The logarithm and sine/cosine are written here from textbook series:
//   ln(w 2^-32): w = 2^e m, m in [sqrt(1/2), sqrt(2)], ln m = 2 atanh(z),
//     z = (m-1)/(m+1), atanh z = sum_{k=0..10} z^(2k+1)/(2k+1), plus
//     (e-32) ln 2 split into a 24-bit head and a tail (Cody and Waite);
//   sin x, cos x on [0, pi/4]: Maclaurin series through x^15 and x^16 in
//     nested form; quadrant and octant reduction of 2 pi u2 are exact because
//     u2 is a multiple of 2^-32.
#pragma once

#include <stdint.h>

namespace wl_bm {

__device__ __forceinline__ double pow2d(int k) // 2^k for |k| < 1000
{
    return __longlong_as_double((long long)(1023 + k) << 52);
}

__device__ inline double log_w(uint64_t w)
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
__device__ inline void sincos_quarter(double g, double &s, double &c)
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

__device__ inline void box_muller(uint32_t u1, uint32_t u2, float &a, float &b)
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

} // namespace wl_bm
