"""Pins for the per-pass addressing parameters (Eq. 1, Eq. 2; Sections 3, 7, 8).

The paper's requirements are checked directly: every stride is odd, > 1,
distinct within a pass and coprime to N (Eq. 2), so that j -> alpha j + gamma
mod N is a permutation (checked by brute force); offsets are uniform on
{0..N-1}.
"""
import math

import numpy as np
import pytest

CAND4 = (3, 5, 9, 15, 45)          # odd divisors > 1 of 45
CAND8 = (3, 5, 7, 9, 15, 21, 35, 45, 63, 105, 315)   # odd divisors > 1 of 315


def _check(n, N, alpha, gamma):
    assert len(set(int(a) for a in alpha)) == n
    for a, g in zip(alpha, gamma):
        a, g = int(a), int(g)
        assert a > 1 and a % 2 == 1
        assert math.gcd(a, N) == 1
        assert 0 <= g < N
        idx = (a * np.arange(N, dtype=np.int64) + g) % N
        assert np.array_equal(np.sort(idx), np.arange(N))   # Eq. 2 -> permutation


@pytest.mark.parametrize("n", [4, 8])
@pytest.mark.parametrize("N", [4, 9, 16, 105, 256, 315, 1000, 3465, 4096, 65536 + 3, 255255])
def test_params_satisfy_paper_constraints(orc, n, N):
    s = orc.seed_state(N * 31 + n)
    for _ in range(20):
        alpha, gamma, s2 = orc.draw_params(n, N, s)
        _check(n, N, alpha, gamma)
        u, s3 = orc.lcg_stream(s, 2 * n)      # exactly 2n uniforms per pass
        assert s2 == s3
        s = s2


def test_power_of_two_strides_are_ordered_choices_from_divisors_of_45(orc):
    """For N coprime to 45 every ordered choice of 4 distinct strides from
    {3,5,9,15,45} is equally likely (120 outcomes), and lcm(strides) = 45."""
    import itertools
    s = orc.seed_state(1)
    counts = {}
    draws = 24000
    for _ in range(draws):
        alpha, gamma, s = orc.draw_params(4, 1 << 20, s)
        key = tuple(int(a) for a in alpha)
        assert all(a in CAND4 for a in key)
        lcm = 1
        for a in key:
            lcm = lcm * a // math.gcd(lcm, a)
        assert lcm == 45
        counts[key] = counts.get(key, 0) + 1
    outcomes = list(itertools.permutations(CAND4, 4))
    assert set(counts) == set(outcomes)
    exp = draws / len(outcomes)
    chi2 = sum((counts[o] - exp) ** 2 / exp for o in outcomes)
    assert chi2 < 119 + 6 * math.sqrt(2 * 119)     # 119 dof


def test_n8_strides_divide_315(orc):
    s = orc.seed_state(2)
    for _ in range(500):
        alpha, _, s = orc.draw_params(8, 1 << 16, s)
        assert all(int(a) in CAND8 for a in alpha)
        assert len(set(int(a) for a in alpha)) == 8


def test_fallback_when_table_exhausted(orc):
    # N divisible by 3 and 5: every candidate shares a factor with N, so the
    # rule takes the smallest free odd numbers coprime to N
    N = 3 * 5 * 7 * 11 * 1000
    alpha, _, _ = orc.draw_params(4, N, orc.seed_state(3))
    assert sorted(int(a) for a in alpha) == [13, 17, 19, 23]
    # N divisible by 3 only: candidate 5, then the fallbacks 7, 11, 13
    alpha, _, _ = orc.draw_params(4, 3 * 4096, orc.seed_state(4))
    assert sorted(int(a) for a in alpha) == [5, 7, 11, 13]


def test_offsets_are_uniform(orc):
    N = 1000
    s = orc.seed_state(2)
    counts = np.zeros(10)
    for _ in range(5000):
        _, gamma, s = orc.draw_params(4, N, s)
        for g in gamma:
            counts[int(g) * 10 // N] += 1
    exp = counts.sum() / 10
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 35   # 9 dof
