"""Pins for the per-pass addressing parameters (Eq. 1, Eq. 2; Sections 3, 7, 8).

The paper's requirements are checked directly: every stride is odd, > 1,
distinct within a pass and coprime to N (Eq. 2), so that j -> alpha j + gamma
mod N is a permutation (checked by brute force); offsets are uniform on
{0..N-1}.
"""
import math

import numpy as np
import pytest

TABLE4 = [(3, 5), (7, 9), (15, 21), (35, 45)]


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


def test_power_of_two_strides_come_from_lcm_bounded_table(orc):
    s = orc.seed_state(1)
    seen = [set() for _ in range(4)]
    for _ in range(400):
        alpha, gamma, s = orc.draw_params(4, 1 << 20, s)
        for i, a in enumerate(alpha):
            assert int(a) in TABLE4[i]
            seen[i].add(int(a))
        lcm = 1
        for a in alpha:
            lcm = lcm * int(a) // math.gcd(lcm, int(a))
        assert 315 % lcm == 0
    assert all(len(x) == 2 for x in seen)   # both choices occur


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
