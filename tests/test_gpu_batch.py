"""Batched generators (one persistent launch for many pools) against the oracle.

Every generator in a batch must produce, bit for bit, what the oracle (and a
single handle) produces for its own n, N, seed and frac: the returned values
of every pass, the pool and the exact sum of squares.  Pool sizes are chosen
to exercise all three per-generator paths: pools kept in shared memory for
all passes, the CTA-local lane-tiled gather (strides with lcm 45), and the
plain gather (N with factors 3 or 5, whose strides fall back).
"""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1004_3114_gb300 import wallace as W  # noqa: E402

NS4 = [4, 16, 100, 256, 1001, 2000, 2100, 3000, 4096, 5000, 8192, 20000, 65536, 100003, 16388, 7]


def _check_batch(orc, b, Ns, seeds, frac, n, runs, mu=0.0, sigma=1.0):
    oracles = [orc.Generator(n, int(N), int(sd), frac) for N, sd in zip(Ns, seeds)]
    for P in runs:
        out = torch.empty(b.out_size(P), dtype=torch.float32, device="cuda")
        b.run(P, out, mu, sigma)
        got = out.cpu().numpy()
        for s, o in enumerate(oracles):
            off = b.out_offset(s, P)
            ref = o.fill(P * int(b.R[s]), mu, sigma)
            assert np.array_equal(got[off:off + ref.size].view(np.uint32), ref.view(np.uint32)), (s, Ns[s], P)
    for s, o in enumerate(oracles):
        assert np.array_equal(b.pool(s).view(np.uint32), o.pool32().view(np.uint32)), (s, Ns[s])
        gs, os_ = b.stats(s), o.stats()
        assert gs.Q == os_.Q and gs.c32 == os_.c32 and gs.passes == os_.passes, (s, Ns[s])
    assert b.sync() == 0


@pytest.mark.parametrize("bulk", [False, True])
def test_batch_n4_mixed_sizes_matches_oracle(orc, bulk):
    seeds = list(range(100, 100 + len(NS4)))
    b = W.Batch(4, NS4, seeds, 1.0)
    if bulk:
        b.set_tuning(0, 2560, 4096)      # the bulk-copy runner
    _check_batch(orc, b, NS4, seeds, 1.0, 4, runs=[3, 2, 1], mu=0.5, sigma=2.0)


@pytest.mark.parametrize("tuning", [(1, 1280, 0), (3, 2560, 8192), (2, 640, 2048), (0, 2560, 4096),
                                    (0, 1280, 0), (0, 2560, 24576)])
def test_batch_tunings_give_identical_streams(orc, tuning):
    """ctas_per_sm = 0: the bulk-copy runner (pools 30000, 65536, 100004,
    16384 and 45060 take the stage ring; 45060 = 2^2 3 5 751 has strides
    from the divisors of 7^2 11, lanes up to 539)."""
    Ns = [300, 2000, 9000, 30000, 65536, 5001, 100004, 16384, 45060]
    seeds = [5, 6, 7, 8, 9, 10, 11, 12, 13]
    b = W.Batch(4, Ns, seeds, 0.5)
    b.set_tuning(*tuning)
    _check_batch(orc, b, Ns, seeds, 0.5, 4, runs=[2, 3])


@pytest.mark.parametrize("tuning", [(0, 2560, 4096), (2, 2560, 2048)])
def test_batch_bulk_runner_any_n_and_lane_count(orc, tuning):
    """The bulk-copy runner on pools of every residue mod 4 (wrapping spans
    shifted past N) and every lane count of the stride sets: 16387 (45 lanes,
    N = 3 mod 4), 16386 = 2 3 2731 (divisors of 175), 20005 = 5 4001 (63),
    17500 = 2^2 5^4 7 (99), 21504 = 2^10 3 7 (275), 16410 = 2 3 5 547 (539)
    and 21000 = 2^3 3 5^3 7 (1573 > 539: the plain gather inside the runner).
    The per-thread runner on the same pools gives the same streams."""
    Ns = [16387, 16386, 20005, 17500, 21504, 16410, 21000, 16389]
    seeds = [21, 22, 23, 24, 25, 26, 27, 28]
    b = W.Batch(4, Ns, seeds, 0.5)
    b.set_tuning(*tuning)
    _check_batch(orc, b, Ns, seeds, 0.5, 4, runs=[2, 3], mu=-1.0, sigma=0.5)


@pytest.mark.parametrize("tuning", [(0, 2560, 2048), (2, 2560, 2048)])
def test_batch_bulk_runner_small_pools(orc, tuning):
    """The bulk-copy runner below N = 16384, where a tile's span of alpha T
    values would exceed N: T is capped at N / max alpha (4096 at 45 lanes: T
    91 of 117; 4098, divisors of 175: T 23, the (lane, time) pair path;
    10005 = 3 5 23 29, 539 lanes: T 18), every residue mod 4, the 63-lane and
    153-lane (5005 = 5 7 11 13: p = 3, q = 17) sets and a plain-gather set
    (8190, lcm 2057).  The per-thread runner on the same pools gives the same
    streams."""
    Ns = [4096, 4099, 4098, 5005, 6010, 8190, 10005, 12289, 4100]
    seeds = [31, 32, 33, 34, 35, 36, 37, 38, 39]
    b = W.Batch(4, Ns, seeds, 1.0)
    b.set_tuning(*tuning)
    _check_batch(orc, b, Ns, seeds, 1.0, 4, runs=[2, 3], mu=0.5, sigma=2.0)


def test_batch_n8(orc):
    Ns = [128, 1000, 3000, 9000]
    seeds = [1, 2, 3, 4]
    b = W.Batch(8, Ns, seeds, 1 / 3)
    _check_batch(orc, b, Ns, seeds, 1 / 3, 8, runs=[2, 2])


def test_batch_without_output_and_autotune_does_not_advance(orc):
    Ns = [512, 4096, 40000, 70000]
    seeds = [11, 12, 13, 14]
    b = W.Batch(4, Ns, seeds, 1.0)
    before = [b.pool(s) for s in range(len(Ns))]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.jsonl")
        t1 = b.autotune(path, 1)
        assert os.path.exists(path)
        t2 = b.autotune(path, 1)       # second call reads the cache
        assert t1 == t2
    for s in range(len(Ns)):
        assert np.array_equal(b.pool(s), before[s])
    b.run(2)                           # values discarded, generators advance
    oracles = [orc.Generator(4, N, sd, 1.0) for N, sd in zip(Ns, seeds)]
    for s, o in enumerate(oracles):
        o.pass_()
        o.pass_()
        assert np.array_equal(b.pool(s).view(np.uint32), o.pool32().view(np.uint32))


def test_config4_all_4096_generators_against_oracle(orc):
    """The batched configuration in full: 4096 generators, n = 4, N
    log-uniform on [2^8, 2^18] (seeded shapes), seeds 0..4095, frac = 1,
    100 passes in one autotuned launch per run (99 passes discarding their
    values, then one pass writing them).  Every generator is checked against
    its own oracle run of the same 100 passes: the returned values of pass
    100, the final pool, Q, S, c, the pass count and the uniform state.  The
    oracle runs go on all host threads (its C calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_1004_3114_gb300.workloads import batch_sizes
    Ns = batch_sizes()
    seeds = np.arange(Ns.size, dtype=np.uint32)
    b = W.Batch(4, Ns, seeds, 1.0)
    b.autotune(None, 2)
    b.run(99, None)
    out = torch.empty(b.out_size(1), dtype=torch.float32, device="cuda")
    b.run(1, out)
    assert b.sync() == 0
    P = 100

    def check(s, got_out, got_pool, gst):
        o = orc.Generator(4, int(Ns[s]), int(seeds[s]), 1.0)
        for _ in range(P):
            o.pass_()
        ref = o.fill(int(b.R[s]))          # the current (100th) pool's returned values
        ost = o.stats()
        ok = (np.array_equal(ref.view(np.uint32), got_out.view(np.uint32))
              and np.array_equal(o.pool32().view(np.uint32), got_pool.view(np.uint32))
              and gst.Q == ost.Q and gst.S == ost.S and gst.c == ost.c and gst.c32 == ost.c32
              and gst.passes == ost.passes == P and gst.lcg == ost.lcg)
        o.close()
        return s, ok

    order = np.argsort(-Ns, kind="stable")      # largest pools first: balanced threads
    with ThreadPoolExecutor() as ex:
        futs = []
        for s in (int(v) for v in order):
            off = b.out_offset(s, 1)
            got_out = out[off:off + int(b.R[s])].cpu().numpy()
            futs.append(ex.submit(check, s, got_out, b.pool(s), b.stats(s)))
        bad = [s for s, ok in (f.result() for f in futs) if not ok]
    assert not bad, f"{len(bad)} of {Ns.size} generators differ, e.g. N = {[int(Ns[s]) for s in bad[:8]]}"
    b.close()


@pytest.mark.parametrize("tuning", [(2, 2560, 2048), (0, 2560, 24576)])
def test_batch_sign_patterns_chi_and_restarts(orc, tuning):
    """wallace_batch_create_ex with WALLACE_MATRIX_SIGNS | WALLACE_CHI_WH (a
    different matrix A D_k each pass, Section 3; Wilson-Hilferty's
    chi-squared sample, Section 4) and wallace_batch_set_restart(4)
    (Section 5): runs of 3, 2 and 5 passes cross the restart points after
    passes 4 and 8.  Every returned value, pool, Q and sign pattern against
    the oracle with the same options, on the per-thread and the bulk-copy
    runners (shared-memory, lane-tiled and plain-gather pools)."""
    mode = W.MATRIX_SIGNS | W.CHI_WH
    Ns = [300, 2000, 9000, 30000, 65536, 5001, 100004, 16384, 45060, 21000]
    seeds = list(range(51, 51 + len(Ns)))
    b = W.Batch(4, Ns, seeds, 0.5, mode=mode)
    b.set_tuning(*tuning)
    b.set_restart(4)
    oracles = [orc.Generator(4, int(N), int(sd), 0.5, mode=orc.FP32 | mode) for N, sd in zip(Ns, seeds)]
    for o in oracles:
        o.set_restart(4)
    for P in (3, 2, 5):
        out = torch.empty(b.out_size(P), dtype=torch.float32, device="cuda")
        b.run(P, out, 0.25, 1.5)
        got = out.cpu().numpy()
        for s, o in enumerate(oracles):
            off = b.out_offset(s, P)
            ref = o.fill(P * int(b.R[s]), 0.25, 1.5)
            assert np.array_equal(got[off:off + ref.size].view(np.uint32), ref.view(np.uint32)), (s, Ns[s], P)
    for s, o in enumerate(oracles):
        assert np.array_equal(b.pool(s).view(np.uint32), o.pool32().view(np.uint32)), (s, Ns[s])
        gs, os_ = b.stats(s), o.stats()
        assert gs.Q == os_.Q and gs.c32 == os_.c32 and gs.S == os_.S and gs.signs == os_.signs, (s, Ns[s])
    assert b.sync() == 0
