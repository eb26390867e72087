"""Pins for the n = 2 variant, RANN4 itself (Section 8): strides alpha from
{3, 5} and beta from {7, 11}, uniform offsets, and a rotation through theta
with pi/6 <= |theta| <= pi/3 or 2 pi/3 <= |theta| <= 5 pi/6 selected through
t = tan(theta/2), the chi-squared scale folded into it.

* The rotation against libm (cos 2 atan t, sin 2 atan t), its ranges, the
  uniform choice of range and of t within it.
* Strides: the RANN4 sets for N a power of two, coprimality (Eq. 2)
  otherwise, every index read once.
* A pass against brute force in exact rational arithmetic (dyadic pools and
  coefficients), and sum-of-squares conservation by the real rotation.
* The generator: N(0,1) moments of its output and the chi-squared targets.
"""
import ctypes as C
import math
from fractions import Fraction as F

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")


def rotation(orc, s):
    st = C.c_uint64(s)
    cs, sn = C.c_double(), C.c_double()
    orc.lib().orc_draw_rotation(C.byref(st), C.byref(cs), C.byref(sn))
    return cs.value, sn.value, int(st.value)


def test_rotation_against_libm_and_ranges(orc):
    s = orc.seed_state(31)
    ranges = np.zeros(4)
    ts = [[], []]
    for _ in range(20000):
        u, _ = orc.lcg_stream(s, 1)
        cs, sn, s = rotation(orc, s)
        u = int(u[0])
        r3 = math.sqrt(3.0)
        lo, hi = ((2 - r3, r3 / 3) if not (u >> 30) & 1 else (r3, 2 + r3))
        t = (lo + (hi - lo) * ((u & 0x3FFFFFFF) / 2**30)) * (-1 if u >> 31 else 1)
        assert abs(cs - math.cos(2 * math.atan(t))) < 4e-16
        assert abs(sn - math.sin(2 * math.atan(t))) < 4e-16
        assert abs(cs * cs + sn * sn - 1) < 1e-15
        assert min(abs(cs), abs(sn)) >= 0.5 - 1e-15
        th = abs(math.atan2(sn, cs))
        assert (math.pi / 6 - 1e-12 <= th <= math.pi / 3 + 1e-12 or
                2 * math.pi / 3 - 1e-12 <= th <= 5 * math.pi / 6 + 1e-12)
        ranges[u >> 30] += 1
        ts[(u >> 30) & 1].append((abs(t) - lo) / (hi - lo))
    assert scipy_stats.chisquare(ranges).pvalue > 1e-3
    for x in ts:
        assert scipy_stats.kstest(x, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("N", [256, 1 << 12, 3 * 1024, 15 * 64, 3 * 5 * 7 * 11 * 13])
def test_rann4_strides(orc, N):
    s = orc.seed_state(2, 0)
    seen = {}
    for _ in range(400):
        alpha, gamma, s = orc.draw_params(2, N, s)
        a, b = int(alpha[0]), int(alpha[1])
        assert math.gcd(a, N) == 1 and math.gcd(b, N) == 1 and a != b and a > 1 and b > 1
        assert 0 <= gamma[0] < N and 0 <= gamma[1] < N
        seen[(a, b)] = seen.get((a, b), 0) + 1
        for i, st in ((0, a), (1, b)):
            idx = (st * np.arange(N) + int(gamma[i])) % N
            assert np.unique(idx).size == N
    if N in (256, 1 << 12):
        assert set(seen) == {(3, 7), (3, 11), (5, 7), (5, 11)}
        assert scipy_stats.chisquare(list(seen.values())).pvalue > 1e-3
    if N == 3 * 1024:
        assert {k[0] for k in seen} == {5}
    if N == 15 * 64:
        assert {k[0] for k in seen} == {7} and {k[1] for k in seen} == {11}


@pytest.mark.parametrize("N", [4, 7, 16])
def test_rann4_pass_brute_force_exact(orc, N):
    rng = np.random.default_rng(N)
    for trial in range(4):
        x = rng.integers(-64, 65, 2 * N).astype(np.float32)
        alpha, gamma, _ = orc.draw_params(2, N, orc.seed_state(trial + 3 * N))
        for Cf, Sf in ((F(3, 4), F(1, 2)), (F(-5, 8), F(7, 8))):
            g0 = [F(float(x[(int(alpha[0]) * j + int(gamma[0])) % N])) for j in range(N)]
            g1 = [F(float(x[N + (int(alpha[1]) * j + int(gamma[1])) % N])) for j in range(N)]
            ref = [Cf * g0[j] + Sf * g1[j] for j in range(N)] + [Cf * g1[j] - Sf * g0[j] for j in range(N)]
            y32 = np.empty(2 * N, dtype=np.float32)
            orc.lib().orc_pass_rot32(N, x, y32, np.ascontiguousarray(alpha[:8], dtype=np.int32),
                                     np.ascontiguousarray(gamma[:8], dtype=np.int64), float(Cf), float(Sf))
            y64 = np.empty(2 * N, dtype=np.float64)
            orc.lib().orc_pass_rot64(N, x.astype(np.float64), y64,
                                     np.ascontiguousarray(alpha[:8], dtype=np.int32),
                                     np.ascontiguousarray(gamma[:8], dtype=np.int64), float(Cf), float(Sf))
            assert [F(float(v)) for v in y32] == ref
            assert [F(float(v)) for v in y64] == ref


def test_rann4_generator(orc):
    n, N = 2, 1 << 14
    g = orc.Generator(n, N, 5, 1 / 3)
    out = g.fill(3_000_000).astype(np.float64)
    m = out.size
    assert abs(out.mean()) < 5 / math.sqrt(m)
    assert abs(out.var() - 1) < 5 * math.sqrt(2 / m)
    assert abs(((out - out.mean()) ** 4).mean() / out.var() ** 2 - 3) < 5 * math.sqrt(24 / m)
    st = g.stats()
    assert st.passes > 100 and st.status == 0
    assert abs(st.drift) < 1e-6 and st.rot_c != 0 and st.rot_s != 0
    assert min(abs(st.rot_c), abs(st.rot_s)) >= 0.5 - 1e-15


def test_rann4_rejects_sign_patterns(orc):
    with pytest.raises(ValueError):
        orc.Generator(2, 256, 1, 1.0, mode=orc.FP32 | orc.SIGNS)
