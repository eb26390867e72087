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


def _smallest_free_primes(N, k):
    """The k smallest odd primes not dividing N, by trial division."""
    out, p = [], 3
    while len(out) < k:
        if all(p % d for d in range(3, int(p ** 0.5) + 1, 2)) and N % p:
            out.append(p)
        p += 2
    return out


def _odd_divisors_above_one(M):
    return [d for d in range(3, M + 1, 2) if M % d == 0]


@pytest.mark.parametrize("N", [4, 9, 15, 21, 35, 105, 256, 1000, 1155, 3 * 4096, 5 * 4096, 15015,
                               255255, 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23, 2 ** 40 * 3 ** 5 * 7,
                               3234846615 * 31 * 37 * 41 * 43])
def test_candidates_are_divisors_of_free_primes(orc, N):
    """n = 4: the odd divisors > 1 of p^2 q; n = 8: of p^2 q r; p < q < r the
    smallest odd primes not dividing N.  Brute force over all odd d <= M."""
    p, q, r = _smallest_free_primes(N, 3)
    assert orc.stride_candidates(4, N) == _odd_divisors_above_one(p * p * q)
    assert orc.stride_candidates(8, N) == _odd_divisors_above_one(p * p * q * r)
    assert len(orc.stride_candidates(4, N)) == 5
    assert len(orc.stride_candidates(8, N)) == 11
    for c in orc.stride_candidates(8, N):
        assert math.gcd(c, N) == 1


def test_candidates_reduce_to_fixed_tables(orc):
    for N in (1 << 10, 1 << 24, 1001, 65536 + 3, 4097):
        assert orc.stride_candidates(4, N) == list(CAND4)
    for N in (1 << 10, 1 << 24, 1 << 16, 11 * 13 * 1024):
        assert orc.stride_candidates(8, N) == list(CAND8)


def test_strides_for_n_divisible_by_3_are_ordered_choices(orc):
    """N = 3 * 4096: candidates {5, 7, 25, 35, 175}; every ordered choice of 4
    is equally likely and the lcm divides 175 (the tiled gather's lane count)."""
    import itertools
    N = 3 * 4096
    cand = (5, 7, 25, 35, 175)
    assert orc.stride_candidates(4, N) == list(cand)
    s = orc.seed_state(5)
    counts = {}
    draws = 24000
    for _ in range(draws):
        alpha, gamma, s = orc.draw_params(4, N, s)
        key = tuple(int(a) for a in alpha)
        assert all(a in cand for a in key)
        lcm = 1
        for a in key:
            lcm = lcm * a // math.gcd(lcm, a)
        assert 175 % lcm == 0
        counts[key] = counts.get(key, 0) + 1
    outcomes = list(itertools.permutations(cand, 4))
    assert set(counts) == set(outcomes)
    exp = draws / len(outcomes)
    chi2 = sum((counts[o] - exp) ** 2 / exp for o in outcomes)
    assert chi2 < 119 + 6 * math.sqrt(2 * 119)     # 119 dof


def test_n2_fallback_when_pair_exhausted(orc):
    # N divisible by 3 and 5: neither of RANN4's {3, 5} is coprime to N, so
    # the x stride is the smallest free odd number coprime to N (7) and the
    # y stride the remaining member of {7, 11}
    N = 15 * 1024
    s = orc.seed_state(3)
    for _ in range(50):
        alpha, _, s = orc.draw_params(2, N, s)
        assert [int(a) for a in alpha] == [7, 11]
    # N divisible by 3 only: x stride is always 5
    s = orc.seed_state(4)
    for _ in range(50):
        alpha, _, s = orc.draw_params(2, 3 * 4096, s)
        assert int(alpha[0]) == 5 and int(alpha[1]) in (7, 11)


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
