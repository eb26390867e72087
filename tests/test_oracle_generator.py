"""Pins for a whole oracle generator over many passes.

* Eq. 3: S = (x + sqrt(2 nu - 1))^2 / 2 with x the withheld last pool value;
  over many passes E[S] = nu and Var[S] = 2 nu - 1/2 (Fisher's approximation).
* The pool's sum of squares after each pass equals the previous target S up
  to binary32 rounding (Section 4; drift monitor of Section 8).
* Tuple-sum invariant: A 1 = 1 for A = (2/n)J - I, so the pool's plain sum
  T obeys T_{k+1} = c_k T_k up to rounding.
* Section 6 / Section 8 user call: returned values are the first R values of
  each new pool, the last value is never returned, and splitting a request
  into several calls does not change the stream.
* Corruption check of Section 8: an overwritten pool is detected.
* FP32 mode stays within 1e-5 of FP64 mode after 1000 passes (n=4, N=256).
"""
import math

import numpy as np
import pytest


def test_S_follows_eq3_and_chi2_moments(orc):
    n, N = 4, 256
    nu = n * N
    g = orc.Generator(n, N, 1, 1.0)
    Ss = []
    r = math.sqrt(2 * nu - 1)
    for _ in range(2000):
        g.pass_()
        st = g.stats()
        x = float(g.pool32()[-1])
        assert st.S == ((x + r) * (x + r)) * 0.5
        Ss.append(st.S)
    Ss = np.array(Ss)
    se = math.sqrt((2 * nu - 0.5) / len(Ss))
    assert abs(Ss.mean() - nu) < 5 * se
    v = Ss.var(ddof=1)
    assert abs(v / (2 * nu - 0.5) - 1) < 5 * math.sqrt(2 / len(Ss))


@pytest.mark.parametrize("n", [4, 8])
def test_sum_of_squares_tracks_target(orc, n):
    g = orc.Generator(n, 1024, 3, 0.5)
    S_prev = g.stats().S
    for _ in range(200):
        g.pass_()
        st = g.stats()
        pool = g.pool64()
        ss = float((pool ** 2).sum())
        assert abs(ss / S_prev - 1) < 2e-6
        assert abs(st.q - ss) <= 1e-9 * ss + n * 1024 * 2.0 ** -32
        assert abs(st.drift) < 2e-6 and st.status == 0
        S_prev = st.S


def test_tuple_sum_invariant(orc):
    g = orc.Generator(4, 4096, 5, 1.0)
    for _ in range(50):
        before = g.pool64()
        c = float(g.stats().c32)
        g.pass_()
        after = g.pool64()
        bound = len(before) * 8 * 2.0 ** -24 * float(np.abs(before).max())
        assert abs(after.sum() - c * before.sum()) <= bound


def test_returned_values_are_pool_prefix(orc):
    n, N, frac = 4, 256, 0.3
    g = orc.Generator(n, N, 8, frac)
    R = orc.returned_count(n * N, frac)
    assert R == int(math.floor(frac * n * N))
    out = g.fill(3 * R)
    g2 = orc.Generator(n, N, 8, frac)
    for k in range(3):
        g2.pass_()
        assert np.array_equal(out[k * R:(k + 1) * R], g2.pool32()[:R])
    assert orc.returned_count(1024, 1.0) == 1023   # last value never returned


def test_fill_split_invariance_and_affine_map(orc):
    whole = orc.Generator(4, 256, 1, 1.0).fill(20000)
    g = orc.Generator(4, 256, 1, 1.0)
    parts = [g.fill(k) for k in (1, 0, 1022, 1, 5000, 3, 13973)]
    assert np.array_equal(np.concatenate(parts), whole)
    mu, sigma = np.float32(-2.5), np.float32(3.25)
    mapped = orc.Generator(4, 256, 1, 1.0).fill(20000, mu, sigma)
    assert np.array_equal(mapped, (mu + (sigma * whole).astype(np.float32)).astype(np.float32))


def test_seeds_and_determinism(orc):
    a = orc.Generator(4, 256, 1, 1.0).fill(5000)
    b = orc.Generator(4, 256, 1, 1.0).fill(5000)
    c = orc.Generator(4, 256, 2, 1.0).fill(5000)
    d = orc.Generator(4, 256, 1, 1.0, stream=1).fill(5000)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c) and not np.array_equal(a, d)


def test_corruption_is_detected(orc):
    g = orc.Generator(4, 256, 1, 1.0)
    g.fill(5000)
    assert g.stats().status == 0
    pool = g.pool32()
    pool[17] = np.float32(40.0)      # user wrote over the work area
    g.set_pool32(pool)
    g.pass_()
    assert g.stats().status == orc.ECORRUPT
    g = orc.Generator(4, 256, 1, 1.0)
    pool = g.pool32()
    pool[3] = np.nan
    g.set_pool32(pool)
    g.pass_()
    assert g.stats().status == orc.ECORRUPT


def test_fp32_within_1e5_of_fp64_after_1000_passes(orc):
    g32 = orc.Generator(4, 256, 1, 1.0, mode=orc.FP32)
    g64 = orc.Generator(4, 256, 1, 1.0, mode=orc.FP64)
    o32 = g32.fill(1023 * 1000)
    o64 = g64.fill(1023 * 1000)
    assert g32.stats().passes == 1000
    dev = np.abs(o32.astype(np.float64) - o64)
    assert dev[-1023:].max() <= 1e-5
    assert dev.max() <= 1e-5
    # parameters and uniforms are identical in both modes
    s32, s64 = g32.stats(), g64.stats()
    assert list(s32.alpha) == list(s64.alpha) and s32.lcg == s64.lcg
