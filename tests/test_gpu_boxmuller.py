"""The Box-Muller comparison generator (wallace_boxmuller_fill) against the
oracle: the exact mode bit for bit, the fast binary32 mode within the error
bound derived below, and the exact mode against a Wallace generator's
initial pool."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1004_3114_gb300 import wallace as W  # noqa: E402


def bm(seed, stream, offset, count, mu=0.0, sigma=1.0, exact=True):
    out = torch.full((count,), float("nan"), dtype=torch.float32, device="cuda")
    W.boxmuller_fill(out, seed, stream, offset, mu, sigma, exact)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def same(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("seed,stream,offset,count", [
    (1, 0, 0, 1), (1, 0, 1, 1), (1, 0, 1, 2), (7, 3, 0, 1000), (7, 3, 333, 4097),
    (9, 0, 12345, 65536), (2, 1, 0, (1 << 20) + 3),
])
def test_exact_mode_bit_exact(orc, seed, stream, offset, count):
    assert same(bm(seed, stream, offset, count), orc.boxmuller_stream(seed, stream, offset, count))


def test_exact_mode_affine_map(orc):
    got = bm(5, 0, 11, 5000, mu=2.5, sigma=0.125)
    assert same(got, orc.boxmuller_stream(5, 0, 11, 5000, 2.5, 0.125))


def test_exact_mode_is_the_initial_pool():
    for n, N, seed in [(4, 256, 1), (4, 1 << 16, 7), (8, 3001, 2)]:
        g = W.Wallace(n, N, seed, 0.5)
        assert same(bm(seed, 0, 0, n * N), g.pool())
        g.close()


def test_fast_mode_error_bound(orc):
    """Binary32 mode: relative error of r below ~2e-7 (float rounding of u1 or of
    2^32-1-U1, and one ulp of logf/log1pf), angle error below 5e-8 rad (float
    rounding of the in-quadrant fraction), one ulp of sincospif and two output
    roundings: |dy| <= 3.7e-7 r.  Checked with margin: |dy| <= 1e-6 r."""
    count = 1 << 21
    got = bm(3, 0, 0, count, exact=False).astype(np.float64)
    ref = orc.boxmuller_stream(3, 0, 0, count).astype(np.float64)
    r = np.repeat(np.hypot(ref[0::2], ref[1::2]), 2)
    err = np.abs(got - ref)
    assert np.all(err <= 1e-6 * r + 1e-30), float(np.max(err / np.maximum(r, 1e-30)))


def test_measurement_size_sampled(orc):
    """The launch the benchmark times (2^28 values): windows at the start, the
    middle and the end against the oracle."""
    count = 1 << 28
    out = torch.empty(count, dtype=torch.float32, device="cuda")
    W.boxmuller_fill(out, 11, 0, 0, 0.0, 1.0, True)
    torch.cuda.synchronize()
    for start in (0, count // 2 + 1, count - 999):
        win = out[start:start + 999].cpu().numpy()
        assert same(win, orc.boxmuller_stream(11, 0, start, win.size))
    del out


def test_invalid_arguments():
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    for offset, count in [(-1, 4), (0, -1)]:
        rc = W.lib().wallace_boxmuller_fill(1, 0, offset, out.data_ptr(), count, 0.0, 1.0, 1, None)
        assert rc == W.EINVAL
    assert W.lib().wallace_boxmuller_fill(1, 0, 0, None, 4, 0.0, 1.0, 1, None) == W.EINVAL
    assert W.lib().wallace_boxmuller_fill(1, 0, 0, None, 0, 0.0, 1.0, 1, None) == W.OK
