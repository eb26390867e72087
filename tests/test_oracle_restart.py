"""Pins for the oracle's restart option (Section 5, restarting) and the LCG
jump it uses.

* orc_lcg_jump against stepping and against the modular closed form
  s_m = a^m s + b (a^m - 1)/(a - 1) (mod 2^64), computed in Python integers.
* The refill of restart r is Box-Muller of the uniforms at positions
  [r 2^40, r 2^40 + nu): checked pair by pair from the closed-form state.
* A restarted generator: the passes before the restart are the plain
  generator's, the strides and offsets after it too (the per-pass draws are
  untouched), the pass after a restart starts a new drift history, and
  undoing that pass (A = J/2 - I is its own inverse) recovers the refill.
"""
import numpy as np
import pytest

A, B, M64 = 6364136223846793005, 1442695040888963407, 1 << 64


def closed_form(s0: int, m: int) -> int:
    am = pow(A, m, M64 * (A - 1))
    geo = ((am - 1) // (A - 1)) % M64      # a^m - 1 is a multiple of a - 1
    return (pow(A, m, M64) * s0 + B * geo) % M64


@pytest.mark.parametrize("m", [0, 1, 2, 7, 1000, 65537])
def test_jump_equals_stepping(orc, m):
    s0 = orc.seed_state(77, 3)
    _, s = orc.lcg_stream(s0, m)
    assert int(orc.lib().orc_lcg_jump(s0, m)) == s


@pytest.mark.parametrize("m", [1 << 40, 3 << 40, (1 << 63) + 12345, (1 << 64) - 1])
def test_jump_closed_form(orc, m):
    s0 = orc.seed_state(5, 0)
    assert int(orc.lib().orc_lcg_jump(s0, m)) == closed_form(s0, m)


def test_restart_pool_pairs(orc):
    seed, stream, r, nu = 9, 1, 2, 4096
    pool = np.empty(nu, dtype=np.float32)
    orc.lib().orc_restart_pool(seed, stream, r, nu, pool)
    u, _ = orc.lcg_stream(closed_form(orc.seed_state(seed, stream), r << 40), nu)
    for p in (0, 1, 777, nu // 2 - 1):
        a, b = orc.box_muller(int(u[2 * p]), int(u[2 * p + 1]))
        assert pool[2 * p] == a and pool[2 * p + 1] == b


def undo_pass(pool, n, N, alpha, gamma, c):
    """Invert one pass: y = c A g with A = (2/n)J - I, A^2 = I, so g = A y / c;
    then g_i[j] = x_i[(alpha_i j + gamma_i) mod N] scatters back."""
    y = pool.astype(np.float64).reshape(n, N)
    g = (2.0 / n) * y.sum(axis=0) - y
    g /= c
    x = np.empty_like(g)
    j = np.arange(N)
    for i in range(n):
        x[i, (alpha[i] * j + gamma[i]) % N] = g[i]
    return x.reshape(-1)


def test_restarted_generator(orc):
    n, N, seed, K = 4, 1024, 3, 3
    g = orc.Generator(n, N, seed, 1.0)
    ref = orc.Generator(n, N, seed, 1.0)
    g.set_restart(K)
    for k in range(K):
        g.pass_()
        ref.pass_()
        assert np.array_equal(g.pool32(), ref.pool32())
    c_before = g.stats().c          # the scale pass K+1 would use without a restart
    g.pass_()                        # restart 1, then pass K+1
    ref.pass_()
    gs, rs = g.stats(), ref.stats()
    assert list(gs.alpha[:n]) == list(rs.alpha[:n]) and list(gs.gamma[:n]) == list(rs.gamma[:n])
    assert gs.passes == rs.passes == K + 1
    assert abs(gs.drift) < 1e-6 and not np.array_equal(g.pool32(), ref.pool32())
    refill = np.empty(n * N, dtype=np.float32)
    orc.lib().orc_restart_pool(seed, 0, 1, n * N, refill)
    # the scale after the refill: c^2 = S/Q of the refilled pool, recovered from
    # the pass output's sum of squares (the pass preserves it up to c^2)
    q_out = float((g.pool32().astype(np.float64) ** 2).sum())
    q_in = float((refill.astype(np.float64) ** 2).sum())
    c = np.sqrt(q_out / q_in)
    assert abs(c - c_before) > 1e-9    # a fresh scale, not the old one
    back = undo_pass(g.pool32(), n, N, gs.alpha[:n], gs.gamma[:n], c)
    assert np.max(np.abs(back - refill)) < 1e-5
