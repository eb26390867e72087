"""Parity of the CUDA library (through its C ABI) with the oracle.

Binary32 mode must match the oracle bit for bit: the initial pool, every pass
(pool, exact Q, chi-squared target S, scale c), every returned value, and the
integer parameters.  Binary64-pool mode must match the binary64 oracle bit for
bit as well (same operations, exact order-free sum of squares).

Cases span several tiles and ragged tails: N = 2^8 (whole pool in shared
memory), N not a multiple of 4, N with small odd factors (stride fallback;
in-kernel plain gather), n = 8, and the full 2^24 x 4 pool.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1004_3114_gb300 import wallace as W  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bits(a):
    return np.ascontiguousarray(a).view(np.uint32 if a.dtype == np.float32 else np.uint64)


def assert_same(got, ref, what=""):
    if not np.array_equal(bits(got), bits(ref)):
        bad = np.nonzero(bits(got) != bits(ref))[0]
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {bad[:5]}: "
                             f"got {got[bad[:5]]} ref {ref[bad[:5]]}")


def assert_stats_equal(g, o, what=""):
    gs, os_ = g.stats(), o.stats()
    assert gs.Q == os_.Q, what
    assert gs.S == os_.S and gs.c == os_.c and gs.c32 == os_.c32, what
    assert gs.passes == os_.passes, what
    assert gs.drift == os_.drift, what
    assert gs.lcg == os_.lcg, what     # uniform state after drawing the next pass's strides
    assert list(gs.alpha[:g.n]) == list(os_.alpha[:g.n]), what
    assert list(gs.gamma[:g.n]) == list(os_.gamma[:g.n]), what
    assert gs.signs == os_.signs, what
    assert gs.rot_c == os_.rot_c and gs.rot_s == os_.rot_s, what
    assert gs.status == os_.status, what


def fill_dev(g, count, mu=0.0, sigma=1.0):
    dt = torch.float32 if g.mode == W.FP32 else torch.float64
    out = torch.empty(count, dtype=dt, device="cuda")
    g.fill(out, mu, sigma)
    return out.cpu().numpy()


@pytest.mark.parametrize("n,N,seed,mode", [
    (4, 256, 1, 0), (4, 1001, 2, 0), (8, 128, 3, 0), (4, 1 << 16, 4, 0), (4, 4, 5, 0),
    (4, 4097, 6, 1), (8, 130, 7, 1),
])
def test_initial_pool_bit_exact(orc, n, N, seed, mode):
    g = W.Wallace(n, N, seed, 1.0, mode=mode)
    o = orc.Generator(n, N, seed, 1.0, mode=mode)
    if mode == 0:
        assert_same(g.pool(), o.pool32(), "pool0")
    else:
        assert_same(g.pool64(), o.pool64(), "pool0")
    assert_stats_equal(g, o, "init")


@pytest.mark.parametrize("variant", [W.VARIANT_AUTO, W.VARIANT_GATHER])
def test_small_config_1000_passes(orc, variant):
    """n=4, N=256, seed 1, frac=1: 1000 passes, every returnable value."""
    g = W.Wallace(4, 256, 1, 1.0)
    g.set_variant(variant)
    o = orc.Generator(4, 256, 1, 1.0)
    got = fill_dev(g, 1023 * 1000)
    ref = o.fill(1023 * 1000)
    assert_same(got, ref, "returned stream")
    assert_same(g.pool(), o.pool32(), "pool after 1000 passes")
    assert_stats_equal(g, o, "after 1000 passes")
    # and the stored oracle snapshot
    with open(os.path.join(GOLDEN, "n4_N256_seed1_frac1.json")) as f:
        snap = json.load(f)["snapshots"][-1]
    assert snap["passes"] == 1000
    assert [int(v) for v in g.pool()[:16].view(np.uint32)] == snap["pool_head"]
    assert str(g.stats().Q) == snap["Q"]


def test_small_config_fp64_deviation(orc):
    """Binary32 stream vs the binary64 oracle after 1000 passes (<= 1e-5)."""
    g = W.Wallace(4, 256, 1, 1.0)
    got = fill_dev(g, 1023 * 1000).astype(np.float64)
    o64 = orc.Generator(4, 256, 1, 1.0, mode=orc.FP64)
    ref = o64.fill(1023 * 1000)
    dev = np.abs(got - ref)
    assert dev.max() <= 1e-5, dev.max()


@pytest.mark.parametrize("n,N,frac,variant", [
    (4, 16384, 1.0, W.VARIANT_TILED),
    (4, 16384, 1.0, W.VARIANT_TILED_ASYNC),
    (4, 1 << 17, 0.5, W.VARIANT_TILED_ASYNC),
    (4, 100004, 1 / 3, W.VARIANT_TILED_TMA),
    (4, 1 << 17, 0.5, W.VARIANT_TILED_TMA),
    (4, 16387, 0.5, W.VARIANT_TILED_TMA),
    (4, 16387, 0.5, W.VARIANT_TILED),
    (4, 20000, 1 / 3, W.VARIANT_TILED),
    (4, 45045, 0.5, W.VARIANT_TILED),      # 3^2 5 7 11 13: fallback strides, in-kernel gather
    (4, 1 << 17, 0.5, W.VARIANT_AUTO),
    (4, 1 << 17, 0.5, W.VARIANT_GATHER),
    (8, 5000, 0.5, W.VARIANT_GATHER),
    (8, 3001, 1.0, W.VARIANT_FUSED),
    (4, 6000, 0.25, W.VARIANT_FUSED),
    (4, 6000, 0.25, W.VARIANT_GATHER),
])
def test_passes_bit_exact(orc, n, N, frac, variant):
    g = W.Wallace(n, N, 11, frac)
    g.set_variant(variant)
    o = orc.Generator(n, N, 11, frac)
    R = g.R
    for k in range(6):
        got = fill_dev(g, R)
        ref = o.fill(R)
        assert_same(got, ref, f"pass {k + 1} output")
        assert_same(g.pool(), o.pool32(), f"pass {k + 1} pool")
        assert_stats_equal(g, o, f"pass {k + 1}")


def test_fill_split_and_affine_map(orc):
    g = W.Wallace(4, 16384, 3, 0.5)
    o = orc.Generator(4, 16384, 3, 0.5)
    sizes = [1, 0, 5, 16383, 16384, 40000, 7, 100001]
    mu, sigma = -3.5, 2.25
    for s in sizes:
        got = fill_dev(g, s, mu, sigma)
        ref = o.fill(s, mu, sigma)
        assert_same(got, ref, f"fill {s}")
    assert_stats_equal(g, o)


def test_explicit_passes_skip_unread_values(orc):
    g = W.Wallace(4, 2048, 8, 1.0)
    o = orc.Generator(4, 2048, 8, 1.0)
    fill_dev(g, 100)
    o.fill(100)
    g.pass_()
    o.pass_()
    assert_same(fill_dev(g, 5000), o.fill(5000), "after explicit pass")


def test_stream_id_and_seeds(orc):
    a = W.Wallace(4, 1024, 9, 1.0, stream_id=0)
    b = W.Wallace(4, 1024, 9, 1.0, stream_id=3)
    ob = orc.Generator(4, 1024, 9, 1.0, stream=3)
    xa, xb = fill_dev(a, 10000), fill_dev(b, 10000)
    assert not np.array_equal(xa, xb)
    assert_same(xb, ob.fill(10000), "stream 3")


@pytest.mark.parametrize("n,N", [(4, 1024), (4, 20000), (8, 2048)])
def test_fp64_pool_mode_bit_exact(orc, n, N):
    g = W.Wallace(n, N, 3, 0.5, mode=W.FP64POOL)
    o = orc.Generator(n, N, 3, 0.5, mode=orc.FP64)
    for k in range(5):
        assert_same(fill_dev(g, g.R, 1.0, 2.0), o.fill(g.R, 1.0, 2.0), f"fp64 pass {k}")
        assert_same(g.pool64(), o.pool64(), f"fp64 pool {k}")
        assert_stats_equal(g, o, f"fp64 pass {k}")


@pytest.mark.parametrize("n,N,frac,variant,mode", [
    (8, 20000, 0.5, W.VARIANT_TWOPHASE, W.FP32),
    (8, 100003, 1 / 3, W.VARIANT_TWOPHASE, W.FP32),
    (8, 1 << 16, 1.0, W.VARIANT_TWOPHASE, W.FP32),
    (8, 9000, 0.25, W.VARIANT_TWOPHASE, W.FP32),      # 3 and 5 divide N: strides up to 7^2 11 13
    (8, 16385, 0.5, W.VARIANT_TWOPHASE, W.FP32),      # N % 4 == 1: blocks that wrap unaligned
    (4, 15 * 4099, 0.5, W.VARIANT_TWOPHASE, W.FP32),  # n = 4, 15 | N: 539 lanes
    (4, 105 * 1001, 1.0, W.VARIANT_TWOPHASE, W.FP32), # 105 | N: strides up to 11^2 13
])
def test_twophase_pass_bit_exact(orc, n, N, frac, variant, mode):
    """The two-phase pass (every sub-vector un-strided into a j-ordered copy,
    then the transform streamed): pools, returned values and every state
    scalar against the oracle, pass by pass."""
    omode = orc.FP32 if mode == W.FP32 else orc.FP64
    g = W.Wallace(n, N, 29, frac, mode=mode)
    g.set_variant(variant)
    o = orc.Generator(n, N, 29, frac, mode=omode)
    for k in range(5):
        assert_same(fill_dev(g, g.R, -2.0, 0.5), o.fill(g.R, -2.0, 0.5), f"pass {k + 1} output")
        if mode == W.FP32:
            assert_same(g.pool(), o.pool32(), f"pass {k + 1} pool")
        else:
            assert_same(g.pool64(), o.pool64(), f"pass {k + 1} pool")
        assert_stats_equal(g, o, f"pass {k + 1}")
    st = g.stats()
    assert st.launches >= 2 * 5   # two kernels a pass
    # fills that start mid-pass: returned values land at unaligned addresses
    for cnt in (1001, 3 * g.R + 5, 7):
        assert_same(fill_dev(g, cnt, 0.25, 3.0), o.fill(cnt, 0.25, 3.0), f"fill of {cnt}")


@pytest.mark.parametrize("N,frac,seed", [
    (16384, 0.5, 29),           # smallest: 7 tiles of 315 lanes x 8 lane times
    (16388, 1 / 3, 5),          # 4 * 17 * 241: spans that wrap at unaligned offsets
    (1 << 16, 1.0, 7),
    (100004, 0.25, 11),         # returned prefix ends inside sub-vector 1
    ((1 << 20) + 12, 0.5, 3),
    ((1 << 21) + 32, 0.5, 19),  # 32 * 65537: a 64 MB+ pool, returned values from a second kernel
    ((1 << 21) + 32, 0.3, 23),
])
@pytest.mark.parametrize("variant", [W.VARIANT_TILED_TMA, W.VARIANT_TILED_CLUSTER, W.VARIANT_TILED])
def test_tma8_pass_bit_exact(orc, N, frac, seed, variant):
    """n = 8 with N coprime to 105: every pass has 315 lanes; the TMA variant
    runs the one-CTA bulk-copy lane-tiled kernel, the cluster variant its
    two-CTA form (tiles of 16 lane times, half-sums exchanged through
    distributed shared memory), and the tiled variant the cluster form for
    pools over 64 MB, else the one-CTA kernel; pools over 64 MB then take the
    returned values' kernel.  Pools, returned values and state scalars
    against the oracle, pass by pass, then fills that start mid-pass."""
    g = W.Wallace(8, N, seed, frac)
    g.set_variant(variant)
    o = orc.Generator(8, N, seed, frac)
    before = g.stats().launches
    for k in range(5):
        assert_same(fill_dev(g, g.R, -2.0, 0.5), o.fill(g.R, -2.0, 0.5), f"pass {k + 1} output")
        assert_same(g.pool(), o.pool32(), f"pass {k + 1} pool")
        assert_stats_equal(g, o, f"pass {k + 1}")
    split = 8 * 4 * N > (64 << 20)
    assert g.stats().launches - before == (10 if split else 5)   # the pass (and its returned values)
    # a pass that returns nothing yet is a single kernel (the two-phase pass takes two)
    before = g.stats().launches
    g.pass_()
    assert g.stats().launches - before == 1
    assert_same(fill_dev(g, g.R, 1.0, 2.0), o.fill(g.R, 1.0, 2.0), "values of a wallace_pass")
    for cnt in (1001, 3 * g.R + 5, 7):
        assert_same(fill_dev(g, cnt, 0.25, 3.0), o.fill(cnt, 0.25, 3.0), f"fill of {cnt}")
    # the two-phase pass stays selectable on the same handle
    g.set_variant(W.VARIANT_TWOPHASE)
    assert_same(fill_dev(g, 2 * g.R), o.fill(2 * g.R), "two-phase after the tiled kernel")


def test_twophase_needs_small_strides(orc):
    """N = 45045 = 3^2 5 7 11 13: n = 8 strides may reach 17^2 19 23 > 16384,
    so no two-phase buffer; AUTO keeps the plain gather (still bit-exact)."""
    g = W.Wallace(8, 45045, 3, 0.5)
    with pytest.raises(W.WallaceError):
        g.set_variant(W.VARIANT_TWOPHASE)
    o = orc.Generator(8, 45045, 3, 0.5)
    for k in range(2):
        assert_same(fill_dev(g, g.R), o.fill(g.R), f"pass {k + 1}")


def test_corruption_detected(orc):
    g = W.Wallace(4, 16384, 1, 0.5)
    fill_dev(g, 3 * g.R)
    assert g.stats().status == 0
    pool = g.pool()
    pool[12345] = np.float32(60.0)     # caller wrote over the work area
    g.set_pool(pool)
    g.pass_()
    assert g.sync() & W.ECORRUPT
    assert g.stats().status & W.ECORRUPT
    g.clear_error()
    assert g.sync() == 0
    h = W.Wallace(4, 256, 1, 1.0)
    pool = h.pool()
    pool[0] = np.nan
    h.set_pool(pool)
    h.pass_()
    assert h.sync() & W.ECORRUPT


def test_fill_host_matches_device(orc):
    g = W.Wallace(4, 16384, 21, 0.5)
    o = orc.Generator(4, 16384, 21, 0.5)
    host = np.empty(3 * g.R + 123, dtype=np.float32)
    g.fill_host(host, 0.5, 1.5)
    assert_same(host, o.fill(host.size, 0.5, 1.5), "fill_host")
    pinned = torch.empty(g.R * 2, dtype=torch.float32).pin_memory()
    g.fill_host(pinned)
    assert_same(pinned.numpy(), o.fill(pinned.numel()), "fill_host pinned")


def test_streams_and_timing(orc):
    s = torch.cuda.Stream()
    g = W.Wallace(4, 1 << 16, 2, 0.5, stream=s)
    g.set_variant(W.VARIANT_TILED)     # one pass kernel per pass
    g.set_timing(True)
    o = orc.Generator(4, 1 << 16, 2, 0.5)
    with torch.cuda.stream(s):
        out = torch.empty(g.R * 3, device="cuda")
        g.fill(out)
    s.synchronize()
    assert_same(out.cpu().numpy(), o.fill(g.R * 3))
    st = g.stats()
    assert st.kernel_launches == 3 and st.kernel_ms > 0
    assert st.launches == 3            # three passes, nothing left to drain first
    g.set_timing(False)
    with torch.cuda.stream(s):
        g.fill(out[: g.R // 2])
        g.fill(out[: g.R])             # drains the rest of the pool, then one pass
    s.synchronize()
    st = g.stats()
    assert st.kernel_launches == 3 and st.launches == 3 + 1 + 2


def stats_equal(gs, os_, n, what=""):
    """Every scalar a pass leaves behind, GPU against oracle."""
    assert gs.Q == os_.Q, what
    assert gs.S == os_.S and gs.c == os_.c and gs.c32 == os_.c32, what
    assert gs.passes == os_.passes and gs.drift == os_.drift, what
    assert gs.lcg == os_.lcg, what
    assert list(gs.alpha[:n]) == list(os_.alpha[:n]), what
    assert list(gs.gamma[:n]) == list(os_.gamma[:n]), what
    assert gs.status == os_.status, what


def test_full_size_200_passes_against_oracle_run(orc):
    """The at-scale configuration end to end: n = 4, N = 2^24 (256 MB pool),
    seed 7, frac = 1/2, 200 passes (Eq. 1 iterated with Eq. 3's rescale).  An
    independent oracle generator runs the same 200 passes on a host thread
    beside the GPU; after every pass the returned values (2^25 of them) are
    compared element by element, and the pass's strides, offsets, uniform
    state, Q, S, c and drift; at the end the whole pool."""
    from concurrent.futures import ThreadPoolExecutor
    n, N, seed, frac, P = 4, 1 << 24, 7, 0.5, 200
    g = W.Wallace(n, N, seed, frac)
    o = orc.Generator(n, N, seed, frac)
    assert_same(g.pool(), o.pool32(), "pool0")
    assert_stats_equal(g, o, "init")
    R = g.R
    out = torch.empty(R, device="cuda")
    host = torch.empty(R, dtype=torch.float32, pin_memory=True)
    refs = [np.empty(R, dtype=np.float32), np.empty(R, dtype=np.float32)]

    def oracle_pass(buf):
        orc.lib().orc_fill32(o._h, buf, R, np.float32(0.0), np.float32(1.0))
        return o.stats()

    with ThreadPoolExecutor(1) as ex:
        fut = ex.submit(oracle_pass, refs[0])
        for k in range(P):
            g.fill(out)
            host.copy_(out)
            gs = g.stats()
            os_ = fut.result()
            if k + 1 < P:
                fut = ex.submit(oracle_pass, refs[(k + 1) & 1])
            assert_same(host.numpy(), refs[k & 1], f"pass {k + 1} returned values")
            stats_equal(gs, os_, n, f"pass {k + 1}")
    assert g.stats().passes == P and g.sync() == 0
    assert_same(g.pool(), o.pool32(), f"pool after {P} passes")
    g.close()
    o.close()


@pytest.mark.parametrize("n,N,variant,mode", [
    (4, 1 << 17, W.VARIANT_TILED_TMA, W.FP32),
    (4, 20000, W.VARIANT_TILED_ASYNC, W.FP32),
    (4, 6000, W.VARIANT_GATHER, W.FP32),
    (8, 3001, W.VARIANT_FUSED, W.FP32),
    (4, 1024, W.VARIANT_AUTO, W.FP64POOL),
])
def test_wilson_hilferty_sample_bit_exact(orc, n, N, variant, mode):
    """The Wilson-Hilferty chi-squared option (Section 4's more accurate
    approximations) through every finaliser: CTA-parallel (TMA pass), last-CTA
    (tiled, gather) and in-kernel (fused), and the binary64 pool."""
    g = W.Wallace(n, N, 13, 0.5, mode=mode | W.CHI_WH)
    g.set_variant(variant)
    o = orc.Generator(n, N, 13, 0.5, mode=(orc.FP32 if mode == W.FP32 else orc.FP64) | orc.CHI_WH)
    assert_stats_equal(g, o, "initial pool")
    for k in range(5):
        got = fill_dev(g, g.R)
        ref = o.fill(g.R)
        assert_same(got, ref, f"pass {k + 1} output")
        assert_stats_equal(g, o, f"pass {k + 1}")


@pytest.mark.parametrize("n,N,variant,mode", [
    (4, 1 << 17, W.VARIANT_TILED_TMA, W.FP32),
    (4, 20000, W.VARIANT_TILED_ASYNC, W.FP32),
    (4, 6000, W.VARIANT_GATHER, W.FP32),
    (8, 3001, W.VARIANT_FUSED, W.FP32),
    (4, 1024, W.VARIANT_AUTO, W.FP64POOL),
])
def test_restart_bit_exact(orc, n, N, variant, mode):
    """Section 5's restart (Box-Muller refill every 2 passes) through every
    pass kernel and the binary64 pool: outputs, pools and state per pass, and
    one fill spanning several restarts."""
    omode = orc.FP32 if mode == W.FP32 else orc.FP64
    g = W.Wallace(n, N, 21, 0.5, mode=mode)
    g.set_variant(variant)
    g.set_restart(2)
    o = orc.Generator(n, N, 21, 0.5, mode=omode)
    o.set_restart(2)
    for k in range(5):
        got = fill_dev(g, g.R)
        ref = o.fill(g.R)
        assert_same(got, ref, f"pass {k + 1} output")
        assert_stats_equal(g, o, f"pass {k + 1}")
        if mode == W.FP32:
            assert_same(g.pool(), o.pool32(), f"pass {k + 1} pool")
    assert_same(fill_dev(g, 5 * g.R + 7), o.fill(5 * g.R + 7), "fill over restarts")
    assert_stats_equal(g, o, "after the long fill")


@pytest.mark.parametrize("n,N,variant,mode", [
    (4, 1 << 17, W.VARIANT_TILED_TMA, W.FP32),
    (4, 16387, W.VARIANT_TILED_TMA, W.FP32),       # N % 4 != 0: the async tiled kernel
    (4, 20000, W.VARIANT_TILED_ASYNC, W.FP32),
    (4, 45045, W.VARIANT_TILED, W.FP32),           # fallback strides: in-kernel gather
    (8, 5000, W.VARIANT_GATHER, W.FP32),
    (8, 20000, W.VARIANT_TWOPHASE, W.FP32),
    (8, 1 << 17, W.VARIANT_TILED_TMA, W.FP32),     # n = 8 bulk-copy kernel, with restarts
    (8, 1 << 17, W.VARIANT_TILED_CLUSTER, W.FP32), # its two-CTA cluster form
    (8, 3001, W.VARIANT_FUSED, W.FP32),
    (4, 1024, W.VARIANT_AUTO, W.FP64POOL),
])
def test_sign_patterns_bit_exact(orc, n, N, variant, mode):
    """A different orthogonal matrix each pass (A D_k, Section 3) through every
    pass kernel and the binary64 pool; combined with the Wilson-Hilferty
    sample and restarts on the TMA case."""
    extra = W.CHI_WH if N == 1 << 17 else 0
    omode = (orc.FP32 if mode == W.FP32 else orc.FP64) | orc.SIGNS | (orc.CHI_WH if extra else 0)
    g = W.Wallace(n, N, 17, 0.5, mode=mode | W.MATRIX_SIGNS | extra)
    g.set_variant(variant)
    o = orc.Generator(n, N, 17, 0.5, mode=omode)
    if extra:
        g.set_restart(3)
        o.set_restart(3)
    seen = set()
    for k in range(7):
        got = fill_dev(g, g.R)
        ref = o.fill(g.R)
        assert_same(got, ref, f"pass {k + 1} output")
        assert_stats_equal(g, o, f"pass {k + 1}")
        seen.add(g.stats().signs)
    assert len(seen) > 1


@pytest.mark.parametrize("N,frac,variant,mode", [
    (256, 1 / 3, W.VARIANT_AUTO, W.FP32),          # shared-memory pool
    (1 << 14, 1 / 3, W.VARIANT_AUTO, W.FP32),      # global-memory gather
    (20000, 1 / 3, W.VARIANT_GATHER, W.FP32),
    (3 * 1024, 0.5, W.VARIANT_AUTO, W.FP32),       # 3 | N: alpha = 5 every pass
    (15 * 64, 1.0, W.VARIANT_GATHER, W.FP32),      # 15 | N: coprimality fallback
    (1 << 12, 1 / 3, W.VARIANT_AUTO, W.FP64POOL),
    (4096, 1 / 3, W.VARIANT_FUSED, W.FP32 | W.CHI_WH),
    (1 << 17, 1 / 3, W.VARIANT_TILED_TMA, W.FP32),  # bulk-copy lane-tiled pass, n = 2
    (100004, 0.5, W.VARIANT_TILED_TMA, W.FP32),
    (16388, 1 / 3, W.VARIANT_AUTO, W.FP32),
    (3 * 16384, 1 / 3, W.VARIANT_TILED_TMA, W.FP32),   # alpha = 5: L = 35 or 55
    (15 * 2048, 1 / 3, W.VARIANT_TILED_TMA, W.FP32),   # strides 7, 11: in-kernel gather
    (1 << 17, 1 / 3, W.VARIANT_TILED_TMA, W.FP32 | W.CHI_WH),
])
def test_rann4_bit_exact(orc, N, frac, variant, mode):
    """RANN4 itself (n = 2, Section 8): strides from {3,5} and {7,11} and a
    rotation drawn each pass, with the scale folded into it."""
    fp = mode & ~W.CHI_WH
    omode = (orc.FP32 if fp == W.FP32 else orc.FP64) | (orc.CHI_WH if mode & W.CHI_WH else 0)
    g = W.Wallace(2, N, 23, frac, mode=mode)
    g.set_variant(variant)
    o = orc.Generator(2, N, 23, frac, mode=omode)
    if mode & W.CHI_WH:
        g.set_restart(4)
        o.set_restart(4)
    assert_stats_equal(g, o, "initial pool")
    for k in range(6):
        got = fill_dev(g, g.R)
        ref = o.fill(g.R)
        assert_same(got, ref, f"pass {k + 1} output")
        assert_stats_equal(g, o, f"pass {k + 1}")
        if fp == W.FP32:
            assert_same(g.pool(), o.pool32(), f"pass {k + 1} pool")
    assert_same(fill_dev(g, 7 * g.R + 5), o.fill(7 * g.R + 5), "long fill")


def test_rann4_rejects_sign_patterns():
    with pytest.raises(W.WallaceError):
        W.Wallace(2, 256, 1, 1.0, mode=W.FP32 | W.MATRIX_SIGNS)


def test_rann4_full_size(orc):
    """RANN4 at its benchmark size (n = 2, N = 2^25, frac = 1/3): three passes
    element by element through the bulk-copy pass."""
    g = W.Wallace(2, 1 << 25, 7, 1 / 3)
    o = orc.Generator(2, 1 << 25, 7, 1 / 3)
    for k in range(3):
        assert_same(fill_dev(g, g.R), o.fill(g.R), f"pass {k + 1} output")
        assert_stats_equal(g, o, f"pass {k + 1}")
    assert_same(g.pool(), o.pool32(), "pool")


@pytest.mark.parametrize("n,N,frac,mode", [
    (4, 16384, 0.5, 0),
    (4, 16387, 1 / 3, 0),            # N = 3 mod 4
    (4, 1 << 16, 0.5, 0),
    (4, 45060, 1.0, 0),              # 2^2 3 5 751: strides from the divisors of 7^2 11
    (4, 21000, 0.5, 0),              # 2^3 3 5^3 7: strides up to 11^2 13
    (4, 1 << 21, 0.25, 0),           # 2^23 values (32 MB), the largest pool it takes
    (8, 1 << 17, 0.5, 0),            # A = J/4 - I
    (8, 3001, 1.0, 0),
    (4, 100003, 0.5, W.MATRIX_SIGNS),   # a sign pattern per pass (A D_k)
    (8, 50000, 0.5, W.MATRIX_SIGNS | W.CHI_WH),
])
def test_l2_multipass_100_passes_bit_exact(orc, n, N, frac, mode):
    """The multi-pass L2 kernel (one cooperative launch per fill, a grid
    barrier per pass): 100 passes in four fills of 25, every returned value,
    the pool and the pass's scalars against the oracle after each fill."""
    g = W.Wallace(n, N, 23, frac, mode=W.FP32 | mode)
    g.set_variant(W.VARIANT_L2RUN)
    o = orc.Generator(n, N, 23, frac, mode=orc.FP32 | mode)
    R = g.R
    for k in range(4):
        st0 = g.stats()
        got = fill_dev(g, 25 * R, -1.25, 0.75)
        assert g.stats().launches - st0.launches == 1, "one launch per fill"
        assert_same(got, o.fill(25 * R, -1.25, 0.75), f"fill {k + 1} values")
        assert_same(g.pool(), o.pool32(), f"pool after {25 * (k + 1)} passes")
        assert_stats_equal(g, o, f"after {25 * (k + 1)} passes")


def test_l2_multipass_split_fills_single_passes_and_grids(orc):
    """Fills that end mid-pass (the rest drained by the next fill), single
    passes through wallace_pass, the Wilson-Hilferty sample, and grids of 1,
    7, 152 and (capped) 100000 CTAs give one stream."""
    n, N = 4, 100004
    g = W.Wallace(n, N, 29, 1 / 3, mode=W.FP32 | W.CHI_WH)
    g.set_variant(W.VARIANT_L2RUN)
    o = orc.Generator(n, N, 29, 1 / 3, mode=orc.FP32 | orc.CHI_WH)
    R = g.R
    for grid, count in ((0, 3 * R + R // 3), (1, R - R // 3 + 5), (7, 4 * R), (152, 2 * R + 17),
                        (100000, 3 * R), (0, 0)):
        g.set_l2_grid(grid)
        assert_same(fill_dev(g, count, 0.5, 2.0), o.fill(count, 0.5, 2.0), f"grid {grid}")
    g.pass_()
    o.pass_()
    g.pass_()
    o.pass_()
    assert_same(g.pool(), o.pool32(), "after single passes")
    assert_stats_equal(g, o, "after single passes")
    assert_same(fill_dev(g, 2 * R), o.fill(2 * R), "fill after single passes")
    assert g.sync() == 0


def test_l2_multipass_refuses_pools_it_cannot_index():
    """Beyond 2^23 values, and n = 2, the variant is refused."""
    for n, N in ((4, (1 << 21) + 4), (2, 1 << 16)):
        g = W.Wallace(n, N, 3, 0.5)
        with pytest.raises(RuntimeError):
            g.set_variant(W.VARIANT_L2RUN)
        g.close()
