"""Pins for the orthogonal transform and one pass (Section 2, Eq. 1; Section 4;
the outlier bound of Section 8).

* A^T A = I exactly, A symmetric, rows with >= 2 nonzeros none small
  (Section 3), read off the oracle's transform applied to unit vectors.
* Sum of squares conserved by the transform up to rounding (Section 2).
* A whole pass against brute force in exact rational arithmetic: explicit
  permutation matrices built from Eq. 1 and a dense A, on dyadic inputs with
  dyadic c where every floating operation is exact.
* Outlier bound: with row 1-norm r (2 for n=4, 5/2 for n=8) and A = A^-1,
  M'/c <= r M and M <= r M'/c.
"""
from fractions import Fraction as F

import numpy as np
import pytest


@pytest.mark.parametrize("n", [4, 8])
def test_transform_matrix_is_orthogonal_symmetric(orc, n):
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n, dtype=np.float64)
        e[k] = 1.0
        M[:, k] = orc.transform64(e, 1.0)
        M32 = orc.transform32(e.astype(np.float32), 1.0)
        assert np.array_equal(M32.astype(np.float64), M[:, k])
    assert np.array_equal(M.T @ M, np.eye(n))        # dyadic entries: exact
    assert np.array_equal(M, M.T)
    assert np.all((M != 0).sum(axis=1) >= 2)
    assert np.abs(M).min() >= 0.25
    assert np.allclose(M @ np.ones(n), np.ones(n))     # A 1 = 1


@pytest.mark.parametrize("n", [4, 8])
def test_transform_conserves_sum_of_squares(orc, n):
    rng = np.random.default_rng(5)
    for _ in range(2000):
        g = rng.standard_normal(n).astype(np.float32)
        y = orc.transform32(g, 1.0).astype(np.float64)
        g64 = g.astype(np.float64)
        assert abs((y ** 2).sum() - (g64 ** 2).sum()) <= 1e-6 * (g64 ** 2).sum() + 1e-30
        c = np.float32(rng.uniform(0.9, 1.1))
        yc = orc.transform32(g, c).astype(np.float64)
        assert abs((yc ** 2).sum() - float(c) ** 2 * (g64 ** 2).sum()) <= 2e-6 * (g64 ** 2).sum() + 1e-30


def _exact_pass(n, N, x, alpha, gamma, c):
    """Eq. 1 by brute force: y = c * (A kron-applied) to the permuted sub-vectors."""
    A = [[F(2, n) - (1 if r == k else 0) for k in range(n)] for r in range(n)]
    xs = [[F(float(x[i * N + j])) for j in range(N)] for i in range(n)]
    # permutation matrices P_i[j][m] = 1 iff m = alpha_i j + gamma_i mod N
    P = []
    for i in range(n):
        Pi = [[0] * N for _ in range(N)]
        for j in range(N):
            Pi[j][(int(alpha[i]) * j + int(gamma[i])) % N] = 1
        P.append(Pi)
    g = [[sum(P[i][j][m] * xs[i][m] for m in range(N)) for j in range(N)] for i in range(n)]
    y = [[c * sum(A[r][k] * g[k][j] for k in range(n)) for j in range(N)] for r in range(n)]
    return [y[i][j] for i in range(n) for j in range(N)]


@pytest.mark.parametrize("n,N", [(4, 4), (4, 8), (4, 9), (4, 16), (8, 5), (8, 8)])
def test_pass_brute_force_exact(orc, n, N):
    rng = np.random.default_rng(100 + N * n)
    for trial in range(4):
        x = rng.integers(-64, 65, n * N).astype(np.float32)
        alpha, gamma, _ = orc.draw_params(n, N, orc.seed_state(trial + 7 * N))
        for c in (F(1), F(3, 4), F(5, 4)):
            ref = _exact_pass(n, N, x, alpha, gamma, c)
            y32 = orc.pass_explicit32(n, N, x, alpha, gamma, float(c))
            y64 = orc.pass_explicit64(n, N, x.astype(np.float64), alpha, gamma, float(c))
            assert [F(float(v)) for v in y32] == ref
            assert [F(float(v)) for v in y64] == ref


def test_pass_rounding_bound(orc):
    n, N = 4, 64
    rng = np.random.default_rng(9)
    x = rng.standard_normal(n * N).astype(np.float32)
    alpha, gamma, _ = orc.draw_params(n, N, orc.seed_state(3))
    c = np.float32(1.0123)
    ref = _exact_pass(n, N, x, alpha, gamma, F(float(c)))
    y = orc.pass_explicit32(n, N, x, alpha, gamma, c)
    scale = np.abs(x).max()
    err = max(abs(F(float(v)) - r) for v, r in zip(y, ref))
    assert float(err) <= 16 * 2.0 ** -24 * scale


@pytest.mark.parametrize("n,r", [(4, 2.0), (8, 2.5)])
def test_outlier_bound(orc, n, r):
    N = 512
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n * N).astype(np.float32)
    s = orc.seed_state(4)
    for _ in range(20):
        alpha, gamma, s = orc.draw_params(n, N, s)
        c = 1.03
        y = orc.pass_explicit32(n, N, x, alpha, gamma, c)
        M, Mp = float(np.abs(x).max()), float(np.abs(y).max())
        assert Mp / c <= r * M * (1 + 1e-6)
        assert M <= r * Mp / c * (1 + 1e-6)
        x = y
