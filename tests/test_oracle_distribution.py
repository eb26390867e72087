"""Distribution checks of the oracle's returned stream (Section 8's tests).

* Moments and Kolmogorov-Smirnov against N(0,1) on 10^7 draws.
* Section 8, first test: pairs (x, y) give u = exp(-(x^2+y^2)/2) ~ U[0,1] and
  v = arctan(x/y) ~ U[-pi/2, pi/2]; 1000 equal bins, chi^2 with 999 dof,
  several seeds and throw-away factors f = 1, 2, 3.
* Section 8, second test: sample mean, second and fourth moments of batches
  compared with their sampling distributions.
"""
import math

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")


def _draws(orc, seed, frac, count, N=1 << 20):
    return orc.Generator(4, N, seed, frac).fill(count).astype(np.float64)


def test_moments_and_ks_1e7(orc):
    x = _draws(orc, 7, 0.5, 10_000_000)
    n = len(x)
    zs = {
        "mean": x.mean() / math.sqrt(1 / n),
        "var": (x.var() - 1) / math.sqrt(2 / n),
        "skew": scipy_stats.skew(x) / math.sqrt(6 / n),
        "kurt": scipy_stats.kurtosis(x) / math.sqrt(24 / n),
    }
    for k, z in zs.items():
        assert abs(z) < 5, (k, z)
    ks = scipy_stats.kstest(x, "norm")
    assert ks.pvalue > 1e-4, ks


@pytest.mark.parametrize("frac", [1.0, 0.5, 1 / 3])
@pytest.mark.parametrize("seed", [1, 2])
def test_paper_uv_chi2(orc, frac, seed):
    x = _draws(orc, seed, frac, 2_000_000, N=1 << 16)
    a, b = x[0::2], x[1::2]
    u = np.exp(-(a * a + b * b) / 2)
    v = np.arctan(a / b)
    for vals, lo, hi in ((u, 0.0, 1.0), (v, -math.pi / 2, math.pi / 2)):
        counts, _ = np.histogram(vals, bins=1000, range=(lo, hi))
        exp = len(vals) / 1000
        chi2 = float(((counts - exp) ** 2 / exp).sum())
        p = scipy_stats.chi2.sf(chi2, 999)
        assert 1e-4 < p < 1 - 1e-4, (chi2, p)


def test_paper_batch_moments(orc):
    x = _draws(orc, 3, 1 / 3, 4_000_000, N=1 << 18)
    batches = x.reshape(40, -1)
    m = batches.shape[1]
    z1 = batches.mean(axis=1) / math.sqrt(1 / m)
    z2 = ((batches ** 2).mean(axis=1) - 1) / math.sqrt(2 / m)
    z4 = ((batches ** 4).mean(axis=1) - 3) / math.sqrt(96 / m)
    for z in (z1, z2, z4):
        assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
