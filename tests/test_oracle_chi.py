"""Pins for the chi-squared samples of Section 4: Eq. 3 (Fisher) and the
Wilson-Hilferty cube (Abramowitz and Stegun 26.4.17), the more accurate
approximation the section points to.

Each pass's S is a function of one pool value x; both maps approximate the
chi-squared quantile function at Phi(x).  The oracle's S is checked against
the exact quantile (scipy) of the same x, its sequence against the
chi-squared law by a Kolmogorov-Smirnov test, and Wilson-Hilferty's implied
law against Fisher's near the centre for a small pool.
"""
import math

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")


def quantile_pairs(orc, n, N, seed, passes, mode):
    """(x_k, S_k) over passes: the withheld last value of each pool and the
    sample the oracle drew from it."""
    g = orc.Generator(n, N, seed, 1.0, mode=mode)
    xs, S = [], []
    for _ in range(passes):
        g.pass_()
        xs.append(float(g.pool32()[-1]))
        S.append(g.stats().S)
    return np.array(xs), np.array(S)


@pytest.mark.parametrize("nu_n,N", [(4, 64), (4, 4096)])
def test_samples_are_chi_squared_quantiles(orc, nu_n, N):
    """S_k against the exact chi-squared quantile of the same normal deviate,
    F^-1(Phi(x_k)) (scipy): Wilson-Hilferty within 2e-4 relative for |x| < 3,
    Eq. 3 within 1e-2; a wrong exponent, sign or scale would miss by far more."""
    nu = nu_n * N
    for mode, tol in ((orc.FP32 | orc.CHI_WH, 2e-4), (orc.FP32, 1e-2)):
        xs, S = quantile_pairs(orc, nu_n, N, 5, 300, mode)
        keep = np.abs(xs) < 3
        exact = scipy_stats.chi2(nu).ppf(scipy_stats.norm.cdf(xs[keep]))
        rel = np.abs(S[keep] / exact - 1)
        assert rel.max() < tol, (mode, rel.max())
        assert keep.sum() > 250


def test_wilson_hilferty_follows_chi_squared(orc):
    n, N = 4, 64
    nu = n * N
    _, S = quantile_pairs(orc, n, N, 6, 2000, orc.FP32 | orc.CHI_WH)
    d, p = scipy_stats.kstest(S, scipy_stats.chi2(nu).cdf)
    assert p > 1e-3, (d, p)


def test_wilson_hilferty_closer_than_fisher_at_the_centre():
    """The implied laws: P(S <= s) = Phi(z(s)) with z the inverse of each map.
    Over the central 98% of chi^2_256, Wilson-Hilferty's CDF error is below
    Fisher's."""
    nu = 256
    a = 2.0 / (9.0 * nu)
    qs = scipy_stats.chi2(nu).ppf(np.linspace(0.01, 0.99, 99))
    wh = scipy_stats.norm.cdf(((qs / nu) ** (1 / 3) - (1 - a)) / math.sqrt(a))
    fi = scipy_stats.norm.cdf(np.sqrt(2 * qs) - math.sqrt(2 * nu - 1))
    true = scipy_stats.chi2(nu).cdf(qs)
    assert np.max(np.abs(wh - true)) < np.max(np.abs(fi - true))
    assert np.max(np.abs(wh - true)) < 1e-4


def test_wilson_hilferty_keeps_the_pool_exact_otherwise(orc):
    """Only S (and hence c) changes: the first pass's strides, offsets and
    initial pool are those of the Eq. 3 generator."""
    g0 = orc.Generator(4, 256, 1, 1.0, mode=orc.FP32)
    g1 = orc.Generator(4, 256, 1, 1.0, mode=orc.FP32 | orc.CHI_WH)
    assert np.array_equal(g0.pool32(), g1.pool32())
    assert g0.stats().Q == g1.stats().Q and g0.stats().S != g1.stats().S
    g0.pass_()
    g1.pass_()
    assert list(g0.stats().alpha[:4]) == list(g1.stats().alpha[:4])
    assert list(g0.stats().gamma[:4]) == list(g1.stats().gamma[:4])
