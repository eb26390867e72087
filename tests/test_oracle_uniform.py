"""Pins for the oracle's subsidiary uniform generator (Section 8: RANN4 takes
its initial pool and per-pass parameters from a seeded uniform generator).

The recurrence is checked against things other than itself: the closed form
of an affine recurrence (geometric series), the full-period property of the
low state bits (Hull-Dobell), invertibility of the seeding mixer, and uniformity.
"""
import numpy as np

A = 6364136223846793005
B = 1442695040888963407
M64 = 1 << 64


def _closed_form_state(s0: int, m: int) -> int:
    # s_m = a^m s_0 + b (a^m - 1) / (a - 1)   (exact integer division over Z)
    am = pow(A, m)
    geo = (am - 1) // (A - 1)
    return (am * s0 + B * geo) % M64


def test_lcg_matches_affine_closed_form(orc):
    s0 = orc.seed_state(12345)
    for m in (1, 2, 3, 17, 1000, 4097):
        u, s = orc.lcg_stream(s0, m)
        assert s == _closed_form_state(s0, m)
        assert int(u[-1]) == s >> 32


def test_lcg_full_period_low_bits(orc):
    # Hull-Dobell: b odd and a = 1 mod 4 give full period 2^64; then the low k
    # bits of the state run through all 2^k residues with period exactly 2^k.
    assert B % 2 == 1 and A % 4 == 1
    k = 12
    s = orc.seed_state(9)
    seen = set()
    import ctypes
    st = ctypes.c_uint64(s)
    first = s & ((1 << k) - 1)
    f = orc.lib().orc_lcg_next
    for step in range(1 << k):
        f(ctypes.byref(st))
        seen.add(st.value & ((1 << k) - 1))
    assert len(seen) == 1 << k
    assert (st.value & ((1 << k) - 1)) == first


def _unxorshift(z: int, k: int) -> int:
    x = z
    for _ in range(64 // k + 1):
        x = z ^ (x >> k)
    return x & (M64 - 1)


def test_splitmix_is_invertible(orc):
    # Each SplitMix64 step (add, xor-shift, multiply by an odd constant) is a
    # bijection on 64-bit words; undo them one by one.
    inv1 = pow(0xbf58476d1ce4e5b9, -1, M64)
    inv2 = pow(0x94d049bb133111eb, -1, M64)
    rng = np.random.default_rng(3)
    for x in [0, 1, 2**63, M64 - 1] + [int(v) for v in rng.integers(0, 2**63, 200)]:
        z = orc.splitmix64(x)
        z = _unxorshift(z, 31)
        z = (z * inv2) % M64
        z = _unxorshift(z, 27)
        z = (z * inv1) % M64
        z = _unxorshift(z, 30)
        assert (z - 0x9e3779b97f4a7c15) % M64 == x


def test_stream_number_changes_sequence(orc):
    # Section 8: the processor number appended to the seed gives different streams.
    a, _ = orc.lcg_stream(orc.seed_state(5, 0), 64)
    b, _ = orc.lcg_stream(orc.seed_state(5, 1), 64)
    c, _ = orc.lcg_stream(orc.seed_state(6, 0), 64)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_uniform_top_bits_are_uniform(orc):
    u, _ = orc.lcg_stream(orc.seed_state(1), 200_000)
    counts = np.bincount(u >> 24, minlength=256)
    exp = len(u) / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # chi^2 with 255 dof: mean 255, sd ~22.6
    assert 150 < chi2 < 380
