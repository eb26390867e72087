"""Pins for the oracle's initial fill (Box-Muller, named by the paper in
Sections 1 and 5 as the way to fill a pool from uniforms).

The project-written logarithm and sine/cosine are checked against the C
library's, and the Box-Muller pair against the textbook formula evaluated
with the C library; the initial pool is checked for N(0,1) moments.
"""
import math

import numpy as np
import pytest


def _ulps(a: float, b: float) -> float:
    return abs(a - b) / math.ulp(max(abs(b), 1e-300))


def test_log_against_libm(orc):
    rng = np.random.default_rng(11)
    ws = [1, 2, 3, 2**31, 2**32 - 1, 2**32, 1518500250, 1518500249, 3037000499, 3037000500]
    ws += [int(w) for w in rng.integers(1, 2**32 + 1, 20000)]
    worst = 0.0
    for w in ws:
        ref = math.log(w / 2**32)      # w / 2^32 is exact in binary64
        got = orc.log_w(w)
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, _ulps(got, ref))
    assert worst <= 2.0, worst


def test_sincos_quarter_against_libm(orc):
    for g in np.linspace(0.0, 0.5, 5001):
        s, c = orc.sincos_quarter(float(g))
        x = float(g) * (math.pi / 2)
        assert abs(s - math.sin(x)) <= 3e-16
        assert abs(c - math.cos(x)) <= 3e-16


def test_sincos_2pi_against_libm(orc):
    rng = np.random.default_rng(12)
    us = [0, 1, 2**29, 2**30, 2**30 + 2**29, 2**31, 3 * 2**30, 2**32 - 1]
    us += [int(u) for u in rng.integers(0, 2**32, 20000)]
    for u in us:
        s, c = orc.sincos_2pi(u)
        th = 2 * math.pi * (u / 2**32)
        assert abs(s - math.sin(th)) <= 2e-15, u
        assert abs(c - math.cos(th)) <= 2e-15, u
        assert abs(s * s + c * c - 1.0) <= 1e-15


def test_box_muller_against_textbook(orc):
    rng = np.random.default_rng(13)
    u1s = rng.integers(0, 2**32, 20000)
    u2s = rng.integers(0, 2**32, 20000)
    worst = 0
    for u1, u2 in zip(u1s, u2s):
        a, b = orc.box_muller(int(u1), int(u2))
        r = math.sqrt(-2.0 * math.log((int(u1) + 1) / 2**32))
        th = 2 * math.pi * (int(u2) / 2**32)
        ra, rb = np.float32(r * math.cos(th)), np.float32(r * math.sin(th))
        for got, ref in ((a, ra), (b, rb)):
            d = abs(int(np.float32(got).view(np.int32)) - int(np.float32(ref).view(np.int32)))
            if np.sign(got) != np.sign(ref) and abs(ref) < 1e-6:
                continue
            worst = max(worst, d)
    assert worst <= 1


def test_box_muller_edge_uniforms(orc):
    # U1 = 2^32 - 1 gives u1 = 1, r = 0: both values are zero
    a, b = orc.box_muller(2**32 - 1, 12345)
    assert a == 0.0 and b == 0.0
    # U1 = 0 gives the largest radius sqrt(64 ln 2)
    a, b = orc.box_muller(0, 0)
    assert abs(a - math.sqrt(64 * math.log(2))) < 1e-5 and b == 0.0


def test_initial_pool_moments(orc):
    g = orc.Generator(4, 1 << 18, 21, 1.0)
    x = g.pool64()
    n = len(x)
    z_mean = x.mean() * math.sqrt(n)
    z_var = (x.var() - 1.0) / math.sqrt(2.0 / n)
    m3 = ((x - x.mean()) ** 3).mean() / x.std() ** 3
    m4 = ((x - x.mean()) ** 4).mean() / x.var() ** 2 - 3.0
    assert abs(z_mean) < 5 and abs(z_var) < 5
    assert abs(m3 / math.sqrt(6.0 / n)) < 5 and abs(m4 / math.sqrt(24.0 / n)) < 5


def test_initial_pool_uses_consecutive_uniform_pairs(orc):
    g = orc.Generator(4, 64, 77, 1.0)
    pool = g.pool32()
    u, _ = orc.lcg_stream(orc.seed_state(77), 256)
    for p in range(128):
        a, b = orc.box_muller(int(u[2 * p]), int(u[2 * p + 1]))
        assert pool[2 * p] == a and pool[2 * p + 1] == b


# ---- the Box-Muller method as a stand-alone generator (the paper's comparison
# method, abstract and Section 1) ----------------------------------------------

def test_boxmuller_stream_is_the_initial_pool(orc):
    """Values [0, nN) of a stream are the initial pool of the Wallace generator
    with the same seed (Sections 5 and 8), itself pinned above to libm."""
    for n, N, seed in [(4, 256, 1), (8, 1001, 9), (4, 4097, 3)]:
        g = orc.Generator(n, N, seed, 1.0)
        assert np.array_equal(orc.boxmuller_stream(seed, 0, 0, n * N).view(np.uint32),
                              g.pool32().view(np.uint32))


def test_boxmuller_stream_pairs_follow_the_uniforms(orc):
    """Pair p uses uniforms 2p and 2p+1 of the (seed, stream) source in order."""
    u, _ = orc.lcg_stream(orc.seed_state(21, 5), 64)
    ref = []
    for p in range(32):
        a, b = orc.box_muller(int(u[2 * p]), int(u[2 * p + 1]))
        ref += [a, b]
    got = orc.boxmuller_stream(21, 5, 0, 64)
    assert np.array_equal(got.view(np.uint32), np.array(ref, dtype=np.float32).view(np.uint32))


@pytest.mark.parametrize("offset,count", [(0, 1), (1, 1), (1, 2), (7, 10), (100, 33), (2, 0)])
def test_boxmuller_stream_windows(orc, offset, count):
    """A window of the stream is the same slice of a longer call."""
    full = orc.boxmuller_stream(4, 2, 0, 200)
    got = orc.boxmuller_stream(4, 2, offset, count)
    assert np.array_equal(got.view(np.uint32), full[offset:offset + count].view(np.uint32))


def test_boxmuller_stream_affine_map(orc):
    """mu + sigma*y is a binary32 multiply then a binary32 add."""
    y = orc.boxmuller_stream(8, 0, 0, 1000)
    mu, sigma = np.float32(-3.25), np.float32(0.7)
    got = orc.boxmuller_stream(8, 0, 0, 1000, float(mu), float(sigma))
    ref = (mu + (sigma * y).astype(np.float32)).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_boxmuller_stream_moments(orc):
    y = orc.boxmuller_stream(12345, 0, 0, 1 << 20).astype(np.float64)
    m = y.size
    assert abs(y.mean()) < 5 / math.sqrt(m)
    assert abs(y.var() - 1.0) < 5 * math.sqrt(2 / m)
    assert abs((y ** 4).mean() - 3.0) < 5 * math.sqrt(96 / m)
