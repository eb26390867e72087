"""Pins for the per-pass sign pattern (Section 3: a different orthogonal
matrix at each pass is preferred; with ORC_SIGNS pass k uses A D_k, D_k a
random diag(+-1)).

* A whole pass with signs against brute force in exact rational arithmetic
  (explicit permutation matrices, dense A, explicit D), dyadic inputs.
* A D is orthogonal for every pattern (read off the pass on unit pools).
* The draws: pass k takes 2n uniforms for its strides and offsets, then one
  for its signs (top n bits); the 2^n patterns come out uniformly.
* The fixed A keeps T_k / sqrt(Q_k) (T the plain sum of the pool) constant
  across passes, a defect of the fixed matrix (A 1 = 1); the sign pattern
  breaks it while keeping Q on its chi-squared targets.
"""
from fractions import Fraction as F

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")


def _exact_pass_signed(n, N, x, alpha, gamma, c, signs):
    A = [[F(2, n) - (1 if r == k else 0) for k in range(n)] for r in range(n)]
    D = [(-1 if (signs >> i) & 1 else 1) for i in range(n)]
    xs = [[F(float(x[i * N + j])) for j in range(N)] for i in range(n)]
    g = [[xs[i][(int(alpha[i]) * j + int(gamma[i])) % N] for j in range(N)] for i in range(n)]
    y = [[c * sum(A[r][k] * D[k] * g[k][j] for k in range(n)) for j in range(N)] for r in range(n)]
    return [y[i][j] for i in range(n) for j in range(N)]


@pytest.mark.parametrize("n,N", [(4, 4), (4, 9), (8, 5), (8, 8)])
def test_signed_pass_brute_force_exact(orc, n, N):
    rng = np.random.default_rng(300 + N * n)
    for trial in range(3):
        x = rng.integers(-64, 65, n * N).astype(np.float32)
        alpha, gamma, _ = orc.draw_params(n, N, orc.seed_state(trial + 11 * N))
        for signs in (0, 1, (1 << n) - 1, int(rng.integers(0, 1 << n))):
            for c in (F(1), F(3, 4)):
                ref = _exact_pass_signed(n, N, x, alpha, gamma, c, signs)
                y32 = orc.pass_explicit32(n, N, x, alpha, gamma, float(c), signs)
                y64 = orc.pass_explicit64(n, N, x.astype(np.float64), alpha, gamma, float(c), signs)
                assert [F(float(v)) for v in y32] == ref
                assert [F(float(v)) for v in y64] == ref


@pytest.mark.parametrize("n", [4, 8])
def test_signed_matrix_orthogonal(orc, n):
    N = 5
    alpha = np.array([1] * n)          # identity addressing isolates the matrix
    gamma = np.zeros(n, dtype=np.int64)
    for signs in range(1 << n):
        M = np.zeros((n, n))
        for k in range(n):
            x = np.zeros(n * N, dtype=np.float64)
            x[k * N] = 1.0
            y = orc.pass_explicit64(n, N, x, alpha, gamma, 1.0, signs)
            M[:, k] = y[0::N]
        assert np.array_equal(M.T @ M, np.eye(n))


def test_sign_draw_order_and_uniformity(orc):
    n, N, seed = 4, 257, 4
    g = orc.Generator(n, N, seed, 1.0, mode=orc.FP32 | orc.SIGNS)
    plain = orc.Generator(n, N, seed, 1.0)
    s = plain.stats().lcg                  # state after the initial pool
    counts = np.zeros(1 << n)
    for k in range(2000):
        g.pass_()
        alpha, gamma, s = orc.draw_params(n, N, s)
        u, s = orc.lcg_stream(s, 1)
        st = g.stats()
        assert list(st.alpha[:n]) == list(alpha[:n]) and list(st.gamma[:n]) == list(gamma[:n])
        assert st.signs == int(u[0]) >> (32 - n)
        counts[st.signs] += 1
    assert scipy_stats.chisquare(counts).pvalue > 1e-3


def test_signs_break_the_fixed_matrix_invariant(orc):
    n, N = 4, 1024
    ratios = {}
    for name, mode in (("fixed", orc.FP32), ("signs", orc.FP32 | orc.SIGNS)):
        g = orc.Generator(n, N, 8, 1.0, mode=mode)
        r = []
        for _ in range(20):
            g.pass_()
            p = g.pool32().astype(np.float64)
            r.append(p.sum() / np.sqrt((p ** 2).sum()))
            assert abs(g.stats().drift) < 1e-5
        ratios[name] = np.array(r)
    fixed, signs = ratios["fixed"], ratios["signs"]
    assert np.max(np.abs(fixed - fixed[0])) < 1e-3 * max(1.0, abs(fixed[0]))
    assert np.std(signs) > 0.3            # T / sqrt(Q) is then roughly N(0, 1)
