"""Distribution checks at the scale of the at-scale single-stream workload:
n = 4, N = 2^24 (2^26-value pool), seed 7, frac = 1/2, output mapped to
N(0, 1); the first 10^8 returned values (three passes).

Mean, variance, skewness and excess kurtosis as z-scores against their
large-sample standard errors under N(0, 1) (sqrt(1/n), sqrt(2/n), sqrt(6/n),
sqrt(24/n)), and the Kolmogorov-Smirnov distance to the N(0, 1) CDF with its
asymptotic p-value.  The statistics are computed with plain torch float64
reductions and a sort on the device (bench.distribution_summary, which the
benchmark line reports too; test infrastructure, not the library).
The stream is bit-exact to the oracle, whose own 10^8 draws give z-scores of
-1.75, -0.11, 0.79, -0.66 and sqrt(n) D = 1.31 for this seed.
"""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_at_scale_stream_moments_and_ks_1e8():
    pytest.importorskip("scipy")
    import bench
    from paper_1004_3114_gb300 import wallace as W
    g = W.Wallace(4, 1 << 24, 7, 0.5)
    out = torch.empty(10 ** 8, dtype=torch.float32, device="cuda")
    g.fill(out)
    assert g.sync() == 0
    s = bench.distribution_summary(out)
    g.close()
    for k in ("mean_z", "var_z", "skew_z", "kurt_z"):
        assert abs(s[k]) < 6.0, s
    assert s["ks_p"] > 1e-4, s
    # the device stream is the oracle's: same statistics to rounding
    assert abs(s["mean_z"] - (-1.747)) < 0.01 and abs(s["ks_sqrt_n_D"] - 1.311) < 0.01, s
