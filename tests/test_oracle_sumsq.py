"""Pins for the exact sum of squares Q (Section 4; the drift monitor of
Section 8).  Each term floor(y^2 2^32) (binary32 pool) or floor(fl(y*y) 2^64)
(binary64 pool) is checked against closed forms and against Python's exact
rational arithmetic; the 128-bit accumulation against Python integers.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest


@pytest.mark.parametrize("y,t", [
    (1.0, 2**32), (-1.0, 2**32), (0.5, 2**30), (1.5, 9 * 2**30), (2.0**-16, 1),
    (2.0**-17, 0), (0.0, 0), (-0.0, 0), (3.0, 9 * 2**32), (255.0, 65025 * 2**32),
])
def test_term32_closed_forms(orc, y, t):
    assert orc.term32(y) == (t, 0)


@pytest.mark.parametrize("y", [256.0, -256.0, 1e30, float("inf"), float("-inf"), float("nan")])
def test_term32_flags_impossible_values(orc, y):
    t, bad = orc.term32(y)
    assert bad == 1 and t == 0


def _exact32(pool):
    return sum(math.floor(F(float(v)) ** 2 * 2**32) for v in pool)


def _exact64(pool):
    # fl(y*y) is the binary64 product, which Python floats compute the same way
    return sum(math.floor(F(float(v) * float(v)) * 2**64) for v in pool)


def test_sumsq32_against_exact_rationals(orc):
    rng = np.random.default_rng(1)
    for scale in (1.0, 1e-3, 30.0):
        pool = (rng.standard_normal(3000) * scale).astype(np.float32)
        pool[:5] = [np.float32(2.0**-149), np.float32(-1e-40), 0.0, np.float32(2**-17), np.float32(1.0)]
        Q, bad = orc.sumsq32(pool)
        assert bad == 0 and Q == _exact32(pool)


def test_sumsq64_against_exact_rationals(orc):
    rng = np.random.default_rng(2)
    for scale in (1.0, 1e-5, 60.0):
        pool = rng.standard_normal(3000) * scale
        Q, bad = orc.sumsq64(pool)
        assert bad == 0 and Q == _exact64(pool)


def test_sumsq_128bit_carry(orc):
    pool = np.full(1 << 17, 255.0, dtype=np.float32)     # 2^17 * 65025 * 2^32 > 2^64
    Q, bad = orc.sumsq32(pool)
    assert bad == 0 and Q == (1 << 17) * 65025 * 2**32 and Q >= 2**64
    pool64 = np.full(1 << 10, 200.0)
    Q, bad = orc.sumsq64(pool64)
    assert Q == (1 << 10) * 40000 * 2**64


def test_sumsq_order_independent(orc):
    rng = np.random.default_rng(3)
    pool = rng.standard_normal(10000).astype(np.float32)
    Q, _ = orc.sumsq32(pool)
    Q2, _ = orc.sumsq32(pool[rng.permutation(len(pool))])
    assert Q == Q2
