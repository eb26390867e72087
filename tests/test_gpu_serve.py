"""The continuous-batching server against the oracle.

Each client's values must be exactly its own generator's stream, whatever
the other clients ask for and however requests are interleaved: every
request's output equals the oracle's fill of the same count, mu and sigma
after that client's earlier requests, and the same client's requests served
alone give the same bytes as in the mix.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1004_3114_gb300 import wallace as W  # noqa: E402


def _mix(seed, n_clients, n_req, max_count):
    rng = np.random.default_rng(seed)
    Ns = np.floor(2.0 ** rng.uniform(6, 15, n_clients)).astype(np.int64)   # 64 .. 32768
    seeds = rng.integers(0, 2**32, n_clients, dtype=np.uint64).astype(np.uint32)
    reqs = [(int(rng.integers(0, n_clients)), int(np.floor(2.0 ** rng.uniform(0, np.log2(max_count)))),
             float(rng.uniform(-3, 3)), float(rng.uniform(0.5, 2))) for _ in range(n_req)]
    return Ns, seeds, reqs


def _serve(Ns, seeds, reqs, frac, budget, tuning=None, interleave=True):
    srv = W.Server(4, Ns, seeds, frac, budget)
    if tuning:
        srv.set_tuning(*tuning)
    ids = []
    for k, (c, cnt, mu, sg) in enumerate(reqs):
        ids.append(srv.submit(c, cnt, mu, sg))
        if interleave and k % 7 == 3:
            srv.progress()          # new requests join while earlier ones run
    srv.drain()
    outs = [srv.result_host(i) for i in ids]
    st = srv.stats()
    assert st.completed == len(reqs) and st.queued == 0 and st.active == 0
    return outs, st


@pytest.mark.parametrize("frac,tuning", [(1 / 3, None), (1.0, (1, 2048, 2)), (0.5, (3, 0, 1)),
                                         (1 / 3, (2, 4096, 0)), (1 / 3, (2, 24576, 0))])
def test_server_outputs_match_oracle(orc, frac, tuning):
    """(2, 24576, 0): pools of up to 24576 values stay in shared memory, those
    above the 256-thread kernel's capacity in the bulk-copy kernel's block."""
    Ns, seeds, reqs = _mix(7, 24, 160, 40000)
    outs, st = _serve(Ns, seeds, reqs, frac, 256 << 20, tuning)
    oracles = {c: orc.Generator(4, int(Ns[c]), int(seeds[c]), frac) for c in set(r[0] for r in reqs)}
    for (c, cnt, mu, sg), got in zip(reqs, outs):
        ref = oracles[c].fill(cnt, np.float32(mu), np.float32(sg))
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), (c, cnt)
    assert st.hbm_peak <= 256 << 20


def test_server_alone_equals_in_mix():
    Ns, seeds, reqs = _mix(11, 16, 120, 30000)
    outs_mix, _ = _serve(Ns, seeds, reqs, 1 / 3, 128 << 20)
    target = reqs[0][0]
    alone = [r for r in reqs if r[0] == target]
    outs_alone, _ = _serve(Ns, seeds, alone, 1 / 3, 128 << 20, interleave=False)
    mix_target = [o for r, o in zip(reqs, outs_mix) if r[0] == target]
    assert len(mix_target) == len(outs_alone) > 1
    for a, b in zip(mix_target, outs_alone):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_server_tight_budget_still_completes(orc):
    """Budget barely above the pools: requests wait for memory, results are
    read and released as they complete, and every value is still exact."""
    Ns = np.array([20000, 30000, 5000, 40000], dtype=np.int64)
    seeds = np.array([1, 2, 3, 4], dtype=np.uint32)
    pools = int(sum(4 * ((N + 8 + 63) // 64 * 64) * 4 for N in Ns))
    reqs = [(k % 4, 150000 + 1000 * k, 0.25, 2.0) for k in range(12)]
    max_out = max(r[1] for r in reqs) * 4
    max_scratch = 4 * ((40000 + 8 + 63) // 64 * 64) * 4
    srv = W.Server(4, Ns, seeds, 0.5, pools + 2 * (max_out + max_scratch) + (1 << 16))
    ids = [srv.submit(c, cnt, mu, sg) for c, cnt, mu, sg in reqs]
    got = {}
    deadline = time.monotonic() + 120.0
    while len(got) < len(ids):
        assert time.monotonic() < deadline, f"only {len(got)} of {len(ids)} requests completed"
        srv.progress()
        for rid in srv.poll():
            got[rid] = srv.result_host(rid)
            srv.release(rid)
    oracles = [orc.Generator(4, int(N), int(sd), 0.5) for N, sd in zip(Ns, seeds)]
    for rid, (c, cnt, mu, sg) in zip(ids, reqs):
        ref = oracles[c].fill(cnt, np.float32(mu), np.float32(sg))
        assert np.array_equal(got[rid].view(np.uint32), ref.view(np.uint32))
    st = srv.stats()
    assert st.hbm_peak <= st.hbm_budget


def test_server_request_larger_than_budget_reports_enomem():
    Ns = np.array([1024, 2048], dtype=np.int64)
    srv = W.Server(4, Ns, np.array([1, 2], dtype=np.uint32), 1.0, 1 << 20)
    srv.submit(0, 1 << 20)          # 4 MB of output cannot fit in a 1 MB budget
    with pytest.raises(W.WallaceError) as e:
        srv.drain()
    assert e.value.code & W.ENOMEM


def test_server_trace_replay_reports_latency():
    Ns = np.floor(2.0 ** np.random.default_rng(3).uniform(10, 16, 64)).astype(np.int64)
    seeds = np.arange(64, dtype=np.uint32)
    srv = W.Server(4, Ns, seeds, 1 / 3, 512 << 20)
    n = 2000
    rng = np.random.default_rng(4)
    arrival = np.cumsum(rng.exponential(1 / 20000.0, n))
    client = rng.integers(0, 64, n).astype(np.int32)
    count = np.floor(2.0 ** rng.uniform(10, 16, n)).astype(np.int64)
    lat = srv.run_trace(arrival, client, count, rng.uniform(-1, 1, n), rng.uniform(0.5, 2, n))
    st = srv.stats()
    assert st.completed == n and np.all(lat > 0) and st.p99_ms >= st.p50_ms > 0
    assert st.values_delivered == int(count.sum())


@pytest.mark.parametrize("ppt", [1, 3])
def test_server_large_pools_split_into_units(orc, ppt):
    """Pools of 2^18..2^20 values run pass-major in several work units per
    pass (tiled and plain-gather strides); every value still exact."""
    Ns = np.array([1 << 16, 1 << 17, 100003, 45045, 70000, 300], dtype=np.int64)
    seeds = np.array([21, 22, 23, 24, 25, 26], dtype=np.uint32)
    srv = W.Server(4, Ns, seeds, 1 / 3, 1 << 30)
    srv.set_tuning(ppt, 4096, 3)
    srv.set_tick(1 << 18, 1 << 20)     # pools above 2^18 values run pass-major
    rng = np.random.default_rng(9)
    reqs = [(int(rng.integers(0, 6)), int(rng.integers(1, 400000)), float(rng.uniform(-2, 2)), 1.5)
            for _ in range(40)]
    ids = []
    for k, (c, cnt, mu, sg) in enumerate(reqs):
        ids.append(srv.submit(c, cnt, mu, sg))
        if k % 5 == 4:
            srv.progress()
    srv.drain()
    oracles = [orc.Generator(4, int(N), int(sd), 1 / 3) for N, sd in zip(Ns, seeds)]
    for rid, (c, cnt, mu, sg) in zip(ids, reqs):
        ref = oracles[c].fill(cnt, np.float32(mu), np.float32(sg))
        assert np.array_equal(srv.result_host(rid).view(np.uint32), ref.view(np.uint32)), (c, cnt)


@pytest.mark.parametrize("ppt", [1, 2])
def test_server_bulk_copy_runner(orc, ppt):
    """ctas_per_sm = 0: requests on pools of 16384..65536 (N % 4 == 0) run the
    bulk-copy runner on the second stream, beside shared-memory pools,
    fallback strides (45060 = 2^2 3 5 751), ragged N and a pool split into
    work units; every value exact."""
    Ns = np.array([16384, 20000, 32768, 65536, 16388, 45060, 300, 3001, 16387, 70000], dtype=np.int64)
    seeds = np.arange(31, 31 + Ns.size, dtype=np.uint32)
    srv = W.Server(4, Ns, seeds, 1 / 3, 1 << 30)
    srv.set_tuning(ppt, 4096, 0)
    rng = np.random.default_rng(12)
    reqs = [(int(rng.integers(0, Ns.size)), int(rng.integers(1, 300000)), float(rng.uniform(-2, 2)),
             float(rng.uniform(0.5, 2))) for _ in range(60)]
    ids = []
    for k, (c, cnt, mu, sg) in enumerate(reqs):
        ids.append(srv.submit(c, cnt, mu, sg))
        if k % 4 == 3:
            srv.progress()
    srv.drain()
    oracles = [orc.Generator(4, int(N), int(sd), 1 / 3) for N, sd in zip(Ns, seeds)]
    for rid, (c, cnt, mu, sg) in zip(ids, reqs):
        ref = oracles[c].fill(cnt, np.float32(mu), np.float32(sg))
        got = srv.result_host(rid)
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), (c, int(Ns[c]), cnt)


@pytest.mark.parametrize("tick", [(1 << 22, 1 << 20), (1 << 22, 1 << 16)])
def test_server_every_pool_on_one_cta(orc, tick):
    """wallace_server_set_tick: every pool (up to 2^22 values) on one CTA per
    request, a tick's share of work per request from 2^16 to 2^20 pool
    values; several ticks in flight on their own streams.  Every value exact."""
    Ns = np.array([1 << 16, 100003, 45060, 3001, 300, 16387, 6000, 1 << 18], dtype=np.int64)
    seeds = np.arange(41, 41 + Ns.size, dtype=np.uint32)
    srv = W.Server(4, Ns, seeds, 1 / 3, 1 << 30)
    srv.set_tuning(2, 24576, 0)
    srv.set_tick(*tick)
    rng = np.random.default_rng(13)
    reqs = [(int(rng.integers(0, Ns.size)), int(rng.integers(1, 600000)), float(rng.uniform(-2, 2)),
             float(rng.uniform(0.5, 2))) for _ in range(60)]
    ids = []
    for k, (c, cnt, mu, sg) in enumerate(reqs):
        ids.append(srv.submit(c, cnt, mu, sg))
        if k % 3 == 2:
            srv.progress()
    srv.drain()
    oracles = [orc.Generator(4, int(N), int(sd), 1 / 3) for N, sd in zip(Ns, seeds)]
    for rid, (c, cnt, mu, sg) in zip(ids, reqs):
        ref = oracles[c].fill(cnt, np.float32(mu), np.float32(sg))
        assert np.array_equal(srv.result_host(rid).view(np.uint32), ref.view(np.uint32)), (c, int(Ns[c]), cnt)


def test_server_sign_patterns_and_restarts(orc):
    """wallace_server_create_ex with WALLACE_MATRIX_SIGNS (a matrix A D_k per
    pass, Section 3) and wallace_server_set_restart(3) (Section 5): a client's
    pool is refilled before the pass after every third of its passes, after
    the values of its current pool still owed have gone out.  Every value
    against the oracle with the same options."""
    Ns = np.array([1 << 16, 100003, 3001, 300, 16387, 6000, 45060], dtype=np.int64)
    seeds = np.arange(61, 61 + Ns.size, dtype=np.uint32)
    srv = W.Server(4, Ns, seeds, 1 / 3, 1 << 30, mode=W.FP32 | W.MATRIX_SIGNS)
    srv.set_tuning(2, 24576, 0)
    srv.set_restart(3)
    rng = np.random.default_rng(17)
    reqs = [(int(rng.integers(0, Ns.size)), int(rng.integers(1, 300000)), float(rng.uniform(-2, 2)),
             float(rng.uniform(0.5, 2))) for _ in range(50)]
    ids = []
    for k, (c, cnt, mu, sg) in enumerate(reqs):
        ids.append(srv.submit(c, cnt, mu, sg))
        if k % 3 == 1:
            srv.progress()
    srv.drain()
    oracles = [orc.Generator(4, int(N), int(sd), 1 / 3, mode=orc.FP32 | orc.SIGNS) for N, sd in zip(Ns, seeds)]
    for o in oracles:
        o.set_restart(3)
    for rid, (c, cnt, mu, sg) in zip(ids, reqs):
        ref = oracles[c].fill(cnt, np.float32(mu), np.float32(sg))
        assert np.array_equal(srv.result_host(rid).view(np.uint32), ref.view(np.uint32)), (c, int(Ns[c]), cnt)
