"""Benchmark: Wallace pool-regeneration pass at scale on one GB300.

Workload (one step = one pass over the whole pool, all of its steps: strided
gather, transform, store, exact sum of squares, chi-squared finaliser with
the next pass's parameter draw, and the returned half of the pool written to
an output buffer in HBM as N(0,1) values):
    n = 4, N = 2^24 (pool of 2^26 binary32 values, 256 MiB, double-buffered),
    A = J/2 - I, seed 7, frac = 1/2 (R = 2^25 values returned per pass).

Prints one JSON line.  `value` is returned N(0,1) variates per second over
all ranks (each rank runs an independent generator, stream id = rank: weak
scaling, no data-path collective).  `--impl reference` times the plain-C
oracle of the same workload on the host cores instead.

On one GPU the line also carries, measured after the timed region, the other
configurations against the plain pass: `batched` (4096 generators in one
launch, every generator checked against its own oracle run), `serve` (the
continuous-batching server under Poisson arrivals: served against offered
values/s, p50/p99), `n8` (A = J/4 - I on the same 2^26-value pool) and
`precision` (binary32 against binary64 pools, 1000 passes).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N(0,1) variates/s, % HBM roofline; batched vs plain pass, oracle bit-exact"
UNIT = "variates/s"
N_SUB, N_LEN, SEED, FRAC = 4, 1 << 24, 7, 0.5
NU = N_SUB * N_LEN
R = int(FRAC * NU)
BYTES_PER_PASS = 8 * NU + 4 * R          # pool read + pool write + returned output
WORKLOAD = (f"Wallace pass, n=4, N=2^24 (2^26-value FP32 pool), A=J/2-I, seed {SEED}, "
            f"frac=1/2 (R=2^25 returned per pass, mu=0 sigma=1, written to HBM)")
PROFILE = os.path.join(ROOT, "profiles", "wl_tma_pass_n4_N2p24.txt")
CLOCK_WINDOW_S = 1.5
KERNEL_SOURCES = ["paper_1004_3114_gb300/csrc/wl_tiled_tma.cu", "paper_1004_3114_gb300/csrc/wl_common.cuh",
                  "paper_1004_3114_gb300/csrc/wl_tma_common.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """dram bytes per launch from the committed ncu summary, if it still
    describes the current kernel source (else None)."""
    try:
        kv = {}
        with open(PROFILE) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_hash():
            return None
        return float(kv["dram_bytes_per_launch_full_size"].split("#")[0])
    except (OSError, KeyError, ValueError):
        return None


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(passes: int):
    """The oracle as it stands (single thread) on the same workload: creation
    excluded, then `passes` passes each returning R values."""
    from oracle import py_oracle as orc
    g = orc.Generator(N_SUB, N_LEN, SEED, FRAC)
    import numpy as np
    out = np.empty(R, dtype=np.float32)
    t0 = time.perf_counter()
    for _ in range(passes):
        orc.lib().orc_fill32(g._h, out, R, np.float32(0.0), np.float32(1.0))
    dt = time.perf_counter() - t0
    g.close()
    return passes * R / dt, dt


def oracle_threads(jobs, threads=None):
    """Run `jobs` (callables that each drive their own oracle generators) on a
    pool of host threads -- the oracle's C calls release the GIL -- and return
    (seconds, threads used)."""
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        for f in [ex.submit(j) for j in jobs]:
            f.result()
    return time.perf_counter() - t0, threads


def batched_cpu_baseline(Ns, seeds, passes: int = 5, every: int = 8):
    """The oracle on a sample of the batched workload (every `every`-th
    generator), one generator per task on all host cores, `passes` passes
    each (creation excluded)."""
    import numpy as np
    from oracle import py_oracle as orc
    pick = list(range(0, len(Ns), every))
    gens = [orc.Generator(4, int(Ns[k]), int(seeds[k]), 1.0) for k in pick]
    Rs = [int(g.stats().R) for g in gens]
    returned = sum(Rs) * passes

    def job(g, r):
        def run():
            out = np.empty(r, dtype=np.float32)
            for _ in range(passes):
                orc.lib().orc_fill32(g._h, out, r, np.float32(0.0), np.float32(1.0))
        return run
    dt, threads = oracle_threads([job(g, r) for g, r in zip(gens, Rs)])
    for g in gens:
        g.close()
    return {"value": returned / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(gens)} of {len(Ns)} generators (one in {every}), {passes} passes each, "
                      f"one generator per task on {threads} threads ({dt:.1f} s, creation excluded)"}


def serve_cpu_baseline(Ns, seeds, tr, n_requests: int = 100):
    """The oracle serving the first `n_requests` requests of the trace: each
    client's requests in arrival order, clients spread over all host cores
    (creation of the clients' generators excluded)."""
    import numpy as np
    from oracle import py_oracle as orc
    by_client = {}
    for k in range(min(n_requests, len(tr["count"]))):
        by_client.setdefault(int(tr["client"][k]), []).append(k)
    gens = {c: orc.Generator(4, int(Ns[c]), int(seeds[c]), 1 / 3) for c in by_client}
    values = int(sum(int(tr["count"][k]) for ks in by_client.values() for k in ks))

    def job(c):
        def run():
            g = gens[c]
            for k in by_client[c]:
                out = np.empty(int(tr["count"][k]), dtype=np.float32)
                orc.lib().orc_fill32(g._h, out, out.size, np.float32(tr["mu"][k]), np.float32(tr["sigma"][k]))
        return run
    dt, threads = oracle_threads([job(c) for c in by_client])
    for g in gens.values():
        g.close()
    return {"value": values / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n_requests} requests ({len(by_client)} clients, {values} values), "
                      f"one client per task on {threads} threads ({dt:.1f} s, creation excluded)"}


def reduce_over_ranks(ms: float, units: int, dist, device) -> tuple[float, int]:
    """Max of the per-rank times and sum of the per-rank units over the
    process group (any backend): the job's time is its slowest rank."""
    if dist is None:
        return ms, units
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def run_reference(args, rank, world):
    if rank != 0:
        return
    # One oracle pass takes about 0.2 s on one host core: the run is bounded
    # by a time budget (at most 2 warm-up passes, then steps until K are done
    # or the budget is spent), and the rate is taken over the steps done.
    warm, steps = min(max(args.warmup, 0), 2), max(args.steps, 1)
    from oracle import py_oracle as orc
    import numpy as np
    g = orc.Generator(N_SUB, N_LEN, SEED, FRAC)
    out = np.empty(R, dtype=np.float32)
    for _ in range(warm):
        orc.lib().orc_fill32(g._h, out, R, np.float32(0.0), np.float32(1.0))
    done = 0
    t0 = time.perf_counter()
    while done < steps and (done == 0 or time.perf_counter() - t0 < args.reference_budget_s):
        orc.lib().orc_fill32(g._h, out, R, np.float32(0.0), np.float32(1.0))
        done += 1
    dt = time.perf_counter() - t0
    value = done * R / dt
    sample = (f"{done} of {steps} steps, each one full oracle pass of the workload "
              f"({dt:.1f} s, budget {args.reference_budget_s:.0f} s; creation excluded), 1 thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": done, "warmup": warm, "ms_per_step": 1e3 * dt / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded generator state; no dataset)",
        "config": {"workload": WORKLOAD, "n": N_SUB, "N": N_LEN, "frac": FRAC,
                   "returned_per_step": R, "oracle": "plain C, FP32 mode, gcc -O2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def distribution_summary(x):
    """z-scores of the first four moments of a 1-D float32 device tensor
    against N(0, 1) (standard errors sqrt(1/n), sqrt(2/n), sqrt(6/n),
    sqrt(24/n)) and its Kolmogorov-Smirnov distance to the N(0, 1) CDF with
    the asymptotic p-value: plain torch float64 reductions and a sort."""
    import torch
    from scipy import special
    n = x.numel()
    xd = x.double()
    m = xd.mean()
    c = xd - m
    v = (c * c).mean()
    skew = (c ** 3).mean() / v ** 1.5
    kurt = (c ** 4).mean() / v ** 2 - 3.0
    del xd, c
    xs = torch.sort(x).values.double()
    F = torch.special.ndtr(xs)
    del xs
    i = torch.arange(1, n + 1, device=x.device, dtype=torch.float64)
    D = float(torch.maximum((i / n - F).max(), (F - (i - 1) / n).max()))
    lam = math.sqrt(n) * D
    return {"draws": n, "mean_z": float(m) / math.sqrt(1 / n), "var_z": (float(v) - 1.0) / math.sqrt(2 / n),
            "skew_z": float(skew) / math.sqrt(6 / n), "kurt_z": float(kurt) / math.sqrt(24 / n),
            "ks_D": D, "ks_sqrt_n_D": lam, "ks_p": float(special.kolmogorov(lam))}


def stream_statistics(draws: int = 10 ** 8):
    """The first `draws` returned values of the benchmark's generator (same
    n, N, seed and frac, stream 0), summarised by distribution_summary."""
    import torch
    from paper_1004_3114_gb300 import wallace as W
    g = W.Wallace(N_SUB, N_LEN, SEED, FRAC)
    out = torch.empty(draws, dtype=torch.float32, device="cuda")
    g.fill(out)
    status = g.sync()
    s = distribution_summary(out)
    s["status"] = int(status)
    g.close()
    del out
    return s


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1004_3114_gb300 import wallace as W

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl", device_id=dev)

    stream = torch.cuda.Stream(device=dev)
    g = W.Wallace(N_SUB, N_LEN, SEED, FRAC, stream_id=rank, stream=stream)
    out = torch.empty(R, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            g.fill(out)
    g.sync()
    torch.cuda.synchronize()

    # Timed region: K back-to-back steps bracketed by two events on the
    # launching stream.  Each step is exactly one pass kernel (the pool's
    # returned values were all handed out by the warm-up), so the kernel's
    # average launch duration is the span over the launch count.  No event
    # sits between two launches: one would stop a pass from starting while
    # the previous one drains (programmatic dependent launch).
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    st0 = g.stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # nvidia-smi samples every 200 ms, longer than the timed region at small
    # K: the sampler runs over a window that opens with the timed region and
    # continues with the same back-to-back passes (untimed) until it has
    # lasted CLOCK_WINDOW_S seconds
    with ClockSampler(local_rank) as clocks:
        t_open = time.perf_counter()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                g.fill(out)
            ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        st1 = g.stats()
        window_passes = 0
        while time.perf_counter() - t_open < CLOCK_WINDOW_S:
            with torch.cuda.stream(stream):
                for _ in range(200):
                    g.fill(out)
            window_passes += 200
            stream.synchronize()
        window_s = time.perf_counter() - t_open
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = st1.launches - st0.launches
    if launches != args.steps:
        raise SystemExit(f"expected one pass kernel per step, saw {launches} launches in {args.steps} steps")
    kernel_ms = ms / launches
    status = g.sync()
    ms, total_units = reduce_over_ranks(ms, args.steps * R, dist, dev)

    # the same kernel timed launch by launch (events around each launch):
    # its isolated duration, without the overlap of consecutive passes
    g.set_timing(True)
    s0 = g.stats()
    with torch.cuda.stream(stream):
        for _ in range(min(args.steps, 200)):
            g.fill(out)
    g.sync()
    s1 = g.stats()
    g.set_timing(False)
    isolated_ms = (s1.kernel_ms - s0.kernel_ms) / max(s1.kernel_launches - s0.kernel_launches, 1)

    # end to end through the C ABI into pinned HOST memory (D2H inside the timed region):
    # one wallace_fill_host call for the values of all timed steps, as a caller
    # streaming values to the host makes it; the call copies each pass's
    # returned values to the host while the next pass runs
    e2e_steps = max(3, min(args.steps, 20))
    host = torch.empty(e2e_steps * R, dtype=torch.float32, pin_memory=True)
    g.fill_host(host[:R])
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    g.fill_host(host)
    e2e_s = time.perf_counter() - t0
    e2e_s, e2e_units = reduce_over_ranks(e2e_s, e2e_steps * R, dist, dev)

    # the other pass kernels on the same pool, for comparison
    cmp = {}
    if rank == 0 and not args.no_compare:
        for name, variant in (("plain_gather", W.VARIANT_GATHER),
                              ("tiled_async_copy", W.VARIANT_TILED_ASYNC)):
            g.set_variant(variant)
            g.set_timing(True)
            s0 = g.stats()
            with torch.cuda.stream(stream):
                for _ in range(20):
                    g.fill(out)
            s1 = g.stats()
            vms = (s1.kernel_ms - s0.kernel_ms) / max(s1.kernel_launches - s0.kernel_launches, 1)
            cmp[name + "_pass_ms"] = vms
            cmp[name + "_GBps"] = BYTES_PER_PASS / (vms * 1e-3) / 1e9
        g.set_variant(W.VARIANT_AUTO)
    g.close()

    if rank == 0:
        peak, peak_kind = hbm_peak()
        achieved = BYTES_PER_PASS / (kernel_ms * 1e-3) / 1e9
        value = total_units / (ms * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator state; no dataset)",
            "config": {"workload": WORKLOAD, "n": N_SUB, "N": N_LEN, "frac": FRAC,
                       "returned_per_step": R, "passes_per_step": 1,
                       "parallelism": f"{world} independent generator(s), stream id = rank",
                       "l2": "inputs larger than L2: 2 x 256 MiB pools + 128 MiB output"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": profiled_traffic(), "kernel": "tma_kernel (lane-tiled pass, bulk copies into a stage ring)",
                         "kernel_ms": kernel_ms, "kernel_ms_isolated": isolated_ms,
                         "timing": "span of the timed region over its launches (one pass kernel per step)",
                         "algorithmic_bytes_per_launch": BYTES_PER_PASS},
            "e2e": {"value": e2e_units / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 4 * R,
                    "call": f"one wallace_fill_host of {e2e_steps} steps' values into pinned host memory"},
            "gpu_launches": int(launches),
            "clocks": dict(clocks.summary(), window_s=window_s, window_passes=args.steps + window_passes,
                           window="the timed region, then the same back-to-back passes untimed"),
            "status": int(status),
        }
        if cmp:
            line["compare"] = cmp
        if not args.no_stats:
            # outside the timed region: moments and KS of the first 10^8 draws
            line["stats"] = stream_statistics()
        if not args.no_cpu_baseline:
            v, dt = cpu_baseline(args.cpu_passes)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"{args.cpu_passes} oracle passes of the same "
                                              f"workload ({dt:.1f} s, creation excluded)"}
        if world == 1 and not args.no_extras:
            # the other configurations, each against the plain pass above
            # (outside the timed region; one GPU)
            plain = value
            b = batched_bench(tune_cache=args.tune_cache, cpu_baseline=not args.no_cpu_baseline)
            b["vs_plain_pass"] = b["value"] / plain
            line["batched"] = b
            torch.cuda.empty_cache()
            sv = serve_bench(cpu_baseline=not args.no_cpu_baseline)
            sv["vs_plain_pass"] = sv["value"] / plain
            line["serve"] = sv
            line["n8"] = n8_bench()
            line["precision"] = precision_study()
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def precision_study(passes: int = 1000, N: int = 1 << 22, seed: int = 3):
    """Binary32 pool (exact integer sum of squares, binary64 scale) against the
    binary64-pool reference mode on the same GPU, same seed and parameters:
    max and RMS deviation after `passes` passes and the per-pass drift
    q_k / S_{k-1} - 1 of each mode."""
    import numpy as np
    import torch  # noqa: F401  (CUDA context)
    from paper_1004_3114_gb300 import wallace as W
    res = {"metric": "precision study", "passes": passes, "N": N, "seed": seed, "cases": []}
    for n in (4, 8):
        g32 = W.Wallace(n, N, seed, 1.0, mode=W.FP32)
        g64 = W.Wallace(n, N, seed, 1.0, mode=W.FP64POOL)
        d32, d64 = [], []
        for _ in range(passes):
            g32.pass_()
            g64.pass_()
            d32.append(g32.stats().drift)
            d64.append(g64.stats().drift)
        p32, p64 = g32.pool64(), g64.pool64()
        dev = np.abs(p32 - p64)
        res["cases"].append({
            "n": n, "max_abs_dev": float(dev.max()), "rms_dev": float(np.sqrt((dev ** 2).mean())),
            "max_abs_value": float(np.abs(p64).max()),
            "fp32_drift_max": float(np.max(np.abs(d32))), "fp32_drift_rms": float(np.sqrt(np.mean(np.square(d32)))),
            "fp64_drift_max": float(np.max(np.abs(d64))),
            "status": [int(g32.sync()), int(g64.sync())]})
        g32.close()
        g64.close()
    return res


def n8_bench(steps: int = 2000, warmup: int = 5, N: int = 1 << 23, frac: float = 0.5, variant: int = 0,
             parity: bool = True) -> dict:
    """n = 8 (A = J/4 - I) on the same 2^26-value pool as the default line
    (N = 2^23, seed 7, frac = 1/2): `steps` back-to-back passes, one step =
    one pass (AUTO: the 315-lane bulk-copy pass on clusters of two CTAs for
    pools over 64 MB, plus the returned values' streaming kernel).  First,
    one pass is compared with the oracle element by element (returned values
    and pool)."""
    import numpy as np
    import torch
    from oracle import py_oracle as orc
    from paper_1004_3114_gb300 import wallace as W
    n = 8
    stream = torch.cuda.Stream()
    g = W.Wallace(n, N, SEED, frac, stream=stream)
    g.set_variant(variant)
    out = torch.empty(g.R, dtype=torch.float32, device="cuda")
    if parity:
        o = orc.Generator(n, N, SEED, frac)
        with torch.cuda.stream(stream):
            g.fill(out)
        got = out.cpu().numpy()
        ref = o.fill(g.R)
        parity = bool(np.array_equal(got.view(np.uint32), ref.view(np.uint32)) and
                      np.array_equal(g.pool().view(np.uint32), o.pool32().view(np.uint32)))
        o.close()
    else:
        parity = None
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            g.fill(out)
    g.sync()
    s0 = g.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            g.fill(out)
        e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    s1 = g.stats()
    status = g.sync()
    peak, kind = hbm_peak()
    bytes_pass = 8 * n * N + 4 * g.R
    achieved = bytes_pass * steps / (ms * 1e-3) / 1e9
    res = {"metric": "n = 8 pass: N(0,1) variates/s", "value": steps * g.R / (ms * 1e-3), "unit": UNIT,
           "workload": f"n=8, N=2^{N.bit_length() - 1}, A=J/4-I, seed {SEED}, frac={frac}",
           "ms_per_pass": ms / steps, "steps": steps, "launches_per_pass": (s1.launches - s0.launches) / steps,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "peak_kind": kind, "algorithmic_bytes_per_pass": bytes_pass},
           "parity_first_pass": parity, "status": int(status)}
    g.close()
    return res


def small_config_bench(passes: int = 1000, reps: int = 20):
    """n = 4, N = 256, seed 1, frac = 1 (R = 1023 returned per pass), mu = 0,
    sigma = 1: one small generator whose pool stays in shared memory, so a
    fill of `passes` passes is one launch; against the oracle on one core."""
    import numpy as np
    import torch
    from oracle import py_oracle as orc
    from paper_1004_3114_gb300 import wallace as W
    n, N, seed = 4, 256, 1
    stream = torch.cuda.Stream()
    g = W.Wallace(n, N, seed, 1.0, stream=stream)
    count = passes * g.R
    out = torch.empty(count, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(3):
            g.fill(out)
    g.sync()
    s0 = g.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            g.fill(out)
        e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    s1 = g.stats()
    status = g.sync()
    g.close()
    nu, R = n * N, int(s1.R)
    o = orc.Generator(n, N, seed, 1.0)
    host = np.empty(count, dtype=np.float32)
    t0 = time.perf_counter()
    for _ in range(reps):
        orc.lib().orc_fill32(o._h, host, count, np.float32(0.0), np.float32(1.0))
    cpu_s = time.perf_counter() - t0
    o.close()
    total_passes = reps * passes
    print(json.dumps({
        "metric": "small-pool generator: N(0,1) variates/s", "value": total_passes * R / (ms * 1e-3),
        "unit": UNIT, "workload": f"n={n}, N={N}, seed {seed}, frac=1 (R={R}), mu=0, sigma=1; "
                                  f"{reps} fills of {passes} passes",
        "us_per_pass": 1e3 * ms / total_passes,
        "launches_per_fill": (s1.launches - s0.launches) / reps,
        "bytes_per_pass": {"algorithmic": 8 * nu + 4 * R, "dram": 4 * R,
                           "note": "the pool stays in shared memory for a whole fill; only the "
                                   "returned values reach HBM"},
        "bound": "latency (one CTA, passes in sequence)",
        "cpu_baseline": {"value": total_passes * R / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"the same {reps} fills ({cpu_s:.2f} s)"},
        "status": int(status)}), flush=True)


def boxmuller_bench(count: int = 1 << 28, reps: int = 20):
    """The Box-Muller comparison generator (the paper's competitor method):
    `reps` launches of `count` values each, binary32 (fast) and binary64
    (exact) arithmetic, beside the Wallace pass at frac = 1/2 and frac = 1 on
    the default pool (n = 4, N = 2^24)."""
    import numpy as np
    import torch
    from oracle import py_oracle as orc
    from paper_1004_3114_gb300 import wallace as W
    stream = torch.cuda.Stream()
    out = torch.empty(count, dtype=torch.float32, device="cuda")
    res = {}
    for name, exact in (("fast", False), ("exact", True)):
        n_reps = reps if not exact else max(2, reps // 10)
        with torch.cuda.stream(stream):
            for _ in range(2):
                W.boxmuller_fill(out, 1, 0, 0, 0.0, 1.0, exact, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(n_reps):
                W.boxmuller_fill(out, 1, 0, k * count, 0.0, 1.0, exact, stream)
            e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = {"value": n_reps * count / (ms * 1e-3), "ms_per_launch": ms / n_reps}
    del out
    peak, kind = hbm_peak()
    wal = {}
    for frac in (0.5, 1.0):
        g = W.Wallace(N_SUB, N_LEN, SEED, frac, stream=stream)
        o = torch.empty(g.R, dtype=torch.float32, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(5):
                g.fill(o)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(300):
                g.fill(o)
            e1.record(stream)
        e1.synchronize()
        wal[f"frac_{frac:g}"] = 300 * g.R / (e0.elapsed_time(e1) * 1e-3)
        g.close()
        del o
    m = 1 << 22
    host = np.empty(m, dtype=np.float32)
    t0 = time.perf_counter()
    orc.lib().orc_boxmuller_stream(1, 0, 0, m, np.float32(0.0), np.float32(1.0), host)
    cpu_s = time.perf_counter() - t0
    fast = res["fast"]
    print(json.dumps({
        "metric": "Box-Muller comparison generator: N(0,1) variates/s", "value": fast["value"],
        "unit": UNIT, "workload": f"{reps} launches of {count} values (binary32 logf/log1pf/sincospif), "
                                 f"seed 1, stream 0",
        "roofline": {"bound": "hbm", "achieved": 4 * fast["value"] / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": 4 * fast["value"] / 1e9 / peak, "peak_kind": kind,
                     "algorithmic_bytes_per_value": 4},
        "exact_binary64": res["exact"],
        "wallace_pass_same_box": {"frac_0.5": wal["frac_0.5"], "frac_1": wal["frac_1"],
                                  "workload": "n=4, N=2^24, seed 7, back-to-back single passes"},
        "cpu_baseline": {"value": m / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{m} values of the binary64 Box-Muller stream ({cpu_s:.2f} s)"}}),
          flush=True)


def variant_bench(steps: int = 2000, warmup: int = 5):
    """The other generator forms on the default pool size (2^26 values), one
    pass per step as in the default line: RANN4 itself (n = 2, N = 2^25,
    frac = 1/3 as RANN4's f = 3), and n = 4 with a random sign pattern per
    pass, with the Wilson-Hilferty sample, and with restarts every 1000 N / R
    passes (Section 5); n = 8 (A = J/4 - I) at N = 2^23 (315-lane bulk-copy
    kernel), the same pool through the two-phase pass, and N = 3 2^21 (strides
    up to 5^2 7 11: the two-phase pass is AUTO's choice); and the binary64
    reference pool (plain gather, 16 bytes per pool value)."""
    import torch
    from paper_1004_3114_gb300 import wallace as W
    peak, kind = hbm_peak()
    A = W.VARIANT_AUTO
    cases = [
        ("rann4_n2", 2, 1 << 25, 1 / 3, W.FP32, 0, A),
        ("n4_signs", 4, 1 << 24, 0.5, W.FP32 | W.MATRIX_SIGNS, 0, A),
        ("n4_wilson_hilferty", 4, 1 << 24, 0.5, W.FP32 | W.CHI_WH, 0, A),
        ("n4_restart", 4, 1 << 24, 0.5, W.FP32, -1, A),
        ("n8", 8, 1 << 23, 0.5, W.FP32, 0, A),
        ("n8_cluster", 8, 1 << 23, 0.5, W.FP32, 0, W.VARIANT_TILED_CLUSTER),
        ("n8_twophase", 8, 1 << 23, 0.5, W.FP32, 0, W.VARIANT_TWOPHASE),
        ("n8_N_3x2p21", 8, 3 << 21, 0.5, W.FP32, 0, A),
        ("n4_fp64_pool", 4, 1 << 24, 0.5, W.FP64POOL, 0, A),
    ]
    res = {}
    stream = torch.cuda.Stream()
    for name, n, N, frac, mode, restart, variant in cases:
        g = W.Wallace(n, N, SEED, frac, mode=mode, stream=stream)
        g.set_variant(variant)
        if restart:
            g.set_restart(max(1, (1000 * N) // g.R))
        esize = 8 if mode == W.FP64POOL else 4
        out = torch.empty(g.R, dtype=torch.float64 if esize == 8 else torch.float32, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                g.fill(out)
        g.sync()
        s0 = g.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                g.fill(out)
            e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        s1 = g.stats()
        nu = n * N
        bytes_pass = 2 * esize * nu + esize * g.R
        launches = s1.launches - s0.launches
        res[name] = {"n": n, "N": N, "frac": frac, "value": steps * g.R / (ms * 1e-3),
                     "ms_per_pass": ms / steps, "launches_per_pass": launches / steps,
                     "roofline_frac": bytes_pass * steps / (ms * 1e-3) / 1e9 / peak,
                     "status": int(g.sync())}
        g.close()
        del out
    print(json.dumps({"metric": "generator variants: N(0,1) variates/s", "unit": UNIT, "peak_gbs": peak,
                      "peak_kind": kind, "steps": steps, "cases": res}), flush=True)


def l2_bench(log2_sizes=range(14, 22), frac: float = 0.5, target_ms: float = 150.0,
             grids=(0,), n: int = 4) -> dict:
    """Pools that stay in L2 between passes (n = 4 or 8, nu = 4 2^k, seed 7): the
    multi-pass kernel (every pass of a fill in one cooperative launch)
    against one launch per pass (the lane-tiled pass), each timed over one
    fill of about `target_ms` of passes.
    Rates are in algorithmic bytes (8 nu + 4 R per pass): an "equivalent"
    fraction of the HBM peak, since the pool stays on chip."""
    import torch
    from paper_1004_3114_gb300 import wallace as W
    peak, kind = hbm_peak()
    stream = torch.cuda.Stream()
    res = {}

    def timed(g, passes):
        out = torch.empty(passes * g.R, dtype=torch.float32, device="cuda")
        with torch.cuda.stream(stream):
            g.fill(out[: 3 * g.R])          # warm-up
        g.sync()
        s0 = g.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            g.fill(out)
            e1.record(stream)
        e1.synchronize()
        s1 = g.stats()
        return e0.elapsed_time(e1) / passes, s1.launches - s0.launches, int(g.sync())

    for k in log2_sizes:
        N = (1 << k) * 4 // n
        nu = n * N
        g = W.Wallace(n, N, SEED, frac, stream=stream)
        try:
            g.set_variant(W.VARIANT_TILED)   # one launch per pass (AUTO takes the L2 kernel here)
        except W.WallaceError:
            g.set_variant(W.VARIANT_GATHER)  # n = 8 pools below 2^14 x 8: no tiled kernel
        byt = 8 * nu + 4 * g.R
        # passes for about target_ms at a first estimate of 10 B per ns
        passes = int(max(200, min(20000, target_ms * 1e6 / max(byt / 10.0, 2000.0))))
        row = {"nu": nu, "passes": passes}
        ms, launches, st = timed(g, passes)
        row["per_pass_launch"] = {"ms_per_pass": ms, "launches": launches, "status": st,
                                  "equiv_frac": byt / (ms * 1e-3) / 1e9 / peak}
        for grid in grids:
            g.set_variant(W.VARIANT_L2RUN)
            g.set_l2_grid(grid)
            ms2, launches2, st2 = timed(g, passes)
            row[f"l2run_grid{grid}"] = {
                "ms_per_pass": ms2, "launches": launches2, "status": st2,
                "equiv_frac": byt / (ms2 * 1e-3) / 1e9 / peak, "speedup": ms / ms2}
        g.close()
        res[f"nu=2^{k + 2}"] = row
    return {"metric": "multi-pass L2 kernel vs one launch per pass: ms per pass", "n": n, "frac": frac,
            "peak_gbs": peak, "peak_kind": kind, "sizes": res}


def oracle_skip(g, count: int, chunk: int = 1 << 22):
    """Advance an oracle generator's output stream by `count` values."""
    import numpy as np
    from oracle import py_oracle as orc
    buf = np.empty(min(count, chunk), dtype=np.float32)
    while count > 0:
        k = min(count, buf.size)
        orc.lib().orc_fill32(g._h, buf, k, np.float32(0.0), np.float32(1.0))
        count -= k


def batched_full_parity(b, Ns, seeds, passes: int, out, passes_in_out: int):
    """Every generator of the batch against its own oracle run: after
    `passes` passes, the returned values of the last pass (mu = 0, sigma = 1;
    the last of the `passes_in_out` passes held in `out`), the final pool, Q,
    S, c, the pass count and the uniform state.  Oracle runs on all host
    threads, largest pools first."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from oracle import py_oracle as orc
    t0 = time.perf_counter()

    def check(s, got_out, got_pool, gst):
        o = orc.Generator(4, int(Ns[s]), int(seeds[s]), 1.0)
        for _ in range(passes):
            o.pass_()
        ref = o.fill(int(b.R[s]))
        ost = o.stats()
        ok = (np.array_equal(ref.view(np.uint32), got_out.view(np.uint32))
              and np.array_equal(o.pool32().view(np.uint32), got_pool.view(np.uint32))
              and gst.Q == ost.Q and gst.S == ost.S and gst.c == ost.c and gst.c32 == ost.c32
              and gst.passes == ost.passes == passes and gst.lcg == ost.lcg)
        o.close()
        return ok

    threads = os.cpu_count() or 1
    with ThreadPoolExecutor(threads) as ex:
        futs = []
        for s in (int(v) for v in np.argsort(-np.asarray(Ns), kind="stable")):
            off = b.out_offset(s, passes_in_out) + (passes_in_out - 1) * int(b.R[s])
            futs.append(ex.submit(check, s, out[off:off + int(b.R[s])].cpu().numpy(), b.pool(s),
                                  b.stats(s)))
        good = sum(1 for f in futs if f.result())
    return {"generators": len(Ns), "bit_exact": int(good), "threads": threads,
            "seconds": time.perf_counter() - t0,
            "checked": f"every generator after {passes} passes: returned values of the last pass, "
                       f"final pool, Q, S, c, pass count and uniform state against its own oracle run"}


def serve_sampled_parity(srv, Ns, seeds, tr, k: int = 8, count: int = 1 << 14):
    """After the trace: one more request for k sampled clients, compared value
    by value with the oracle advanced by each client's requests of the trace."""
    import numpy as np
    from oracle import py_oracle as orc
    rng = np.random.default_rng(7)
    clients = [int(c) for c in rng.choice(np.unique(tr["client"]), size=k, replace=False)]
    rids = [srv.submit(c, count, 0.5, 2.0) for c in clients]
    srv.drain()
    got = {c: srv.result_host(r) for c, r in zip(clients, rids)}
    for r in rids:
        srv.release(r)
    ok = {}

    def job(c):
        def run():
            g = orc.Generator(4, int(Ns[c]), int(seeds[c]), 1 / 3)
            oracle_skip(g, int(tr["count"][tr["client"] == c].sum()))
            ref = g.fill(count, 0.5, 2.0)
            ok[c] = bool(np.array_equal(ref.view(np.uint32), got[c].view(np.uint32)))
            g.close()
        return run
    oracle_threads([job(c) for c in clients])
    return {"clients": k, "values_per_client": count, "bit_exact": int(sum(ok.values())),
            "checked": "one request per sampled client after the trace, against the oracle "
                       "advanced by that client's requests"}


def batched_bench(passes_per_run: int = 10, runs: int = 10, seq_passes: int = 2,
                  power_of_two: bool = False, count: int = 4096, tune_cache: str | None = None,
                  cpu_baseline: bool = True) -> dict:
    """4096 generators, n = 4, N log-uniform on [2^8, 2^18], seeds 0..4095,
    frac = 1: `runs` batched launches of `passes_per_run` passes (autotuned,
    CUDA graph), against the same generators run one after another through
    single-generator handles (`seq_passes` passes each)."""
    import numpy as np
    import torch
    from paper_1004_3114_gb300 import wallace as W
    from paper_1004_3114_gb300.workloads import batch_sizes
    Ns = batch_sizes(count=count, power_of_two=power_of_two)
    seeds = np.arange(len(Ns), dtype=np.uint32)
    stream = torch.cuda.Stream()
    b = W.Batch(4, Ns, seeds, 1.0, stream=stream)
    nu_total = int(4 * Ns.sum())
    R_total = int(b.R.sum())
    bytes_per_pass = 8 * nu_total + 4 * R_total
    t0 = time.perf_counter()
    tuning = b.autotune(tune_cache, 2)
    tune_s = time.perf_counter() - t0
    out = torch.empty(b.out_size(passes_per_run), dtype=torch.float32, device="cuda")
    b.run(1, None)   # warm-up (graph instantiation)
    b.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(runs):
            b.run(passes_per_run, out)
        ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    status = b.sync()
    passes = runs * passes_per_run
    value = passes * R_total / (ms * 1e-3)
    peak, kind = hbm_peak()
    achieved = passes * bytes_per_pass / (ms * 1e-3) / 1e9
    # parity of every generator (1 warm-up pass + the timed passes)
    parity = batched_full_parity(b, Ns, seeds, 1 + passes, out, passes_per_run)
    b.close()
    del out
    # the same generators, one handle each, one after another
    handles = [W.Wallace(4, int(N), int(sd), 1.0, stream=stream) for N, sd in zip(Ns, seeds)]
    outs = [torch.empty(seq_passes * h.R, dtype=torch.float32, device="cuda") for h in handles]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for h, o in zip(handles, outs):
            h.fill(o)
        e1.record(stream)
    e1.synchronize()
    seq_ms = e0.elapsed_time(e1)
    seq_value = seq_passes * R_total / (seq_ms * 1e-3)
    for h in handles:
        h.close()
    cpu = batched_cpu_baseline(Ns, seeds) if cpu_baseline else None
    return {
        "metric": "batched generators: N(0,1) variates/s", "value": value, "unit": UNIT,
        "cpu_baseline": cpu,
        "workload": f"{count} generators, n=4, N log-uniform on [2^8, 2^18]"
                    f"{' (powers of two)' if power_of_two else ''}, seeds 0..{count - 1}, frac=1",
        "sum_nu": nu_total, "passes": passes, "runs": runs, "ms": ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": kind,
                     "algorithmic_bytes_per_pass": bytes_per_pass},
        "tuning": {"ctas_per_sm": tuning[0], "etarget": tuning[1], "fused_max": tuning[2],
                   "autotune_s": tune_s},
        "sequential_handles": {"value": seq_value, "passes": seq_passes, "ms": seq_ms,
                               "launches": "one fill per generator"},
        "speedup_vs_sequential": value / seq_value, "parity": parity,
        "status": int(status)}


def lane_count(N: int) -> int:
    """Lanes of the lane-tiled geometry of an n = 4 pool of length N: the lcm
    of any pass's strides, p^2 q for p < q the smallest odd primes not
    dividing N (the stride candidates are the odd divisors of p^2 q).  Used
    only to sort pool sizes into classes."""
    pr = [p for p in (3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61) if N % p][:2]
    return pr[0] * pr[0] * pr[1]


# n4div: 4 divides N; other: it does not; small: N below 2^14 (per-thread paths)
BATCH_CLASSES = {
    "45_lanes_n4div": lambda N: N >= 1 << 14 and lane_count(N) == 45 and N % 4 == 0,
    "45_lanes_other": lambda N: N >= 1 << 14 and lane_count(N) == 45 and N % 4 != 0,
    "63_lanes": lambda N: N >= 1 << 14 and lane_count(N) == 63,
    "175_lanes": lambda N: N >= 1 << 14 and lane_count(N) == 175,
    "539_lanes": lambda N: N >= 1 << 14 and lane_count(N) == 539,
    "over_539_lanes": lambda N: N >= 1 << 14 and lane_count(N) > 539,
    "small": lambda N: N < 1 << 14,
}


def batched_classes_bench(names=None, pools: int = 1024, passes: int = 10, runs: int = 3):
    """The bulk-copy batched runner on one class of pool sizes at a time:
    `pools` generators whose N (log-uniform on [2^14, 2^18], or [2^8, 2^14]
    for the small class, seeded) fall in the class, `runs` timed launches of
    `passes` passes after one warm-up launch; rate in algorithmic bytes."""
    import numpy as np
    import torch
    from paper_1004_3114_gb300 import wallace as W
    peak, kind = hbm_peak()
    res = {}
    for name in names or list(BATCH_CLASSES):
        cond = BATCH_CLASSES[name]
        rng = np.random.default_rng(11)
        lo, hi = (8, 14) if name.startswith("small") else (14, 18)
        Ns = []
        while len(Ns) < pools:
            N = int(2 ** (lo + (hi - lo) * rng.random()))
            if cond(N):
                Ns.append(N)
        Ns = np.array(Ns, dtype=np.int64)
        stream = torch.cuda.Stream()
        b = W.Batch(4, Ns, np.arange(pools, dtype=np.uint32), 1.0, stream=stream)
        b.set_tuning(0, 2560, 2048)
        out = torch.empty(b.out_size(passes), dtype=torch.float32, device="cuda")
        b.run(passes, out)
        b.sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(runs):
                b.run(passes, out)
            ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / (runs * passes)
        status = b.sync()
        nu = int(4 * Ns.sum())
        byt = 8 * nu + 4 * int(b.R.sum())
        res[name] = {"pools": pools, "sum_nu": nu, "ms_per_pass": ms, "TBps": byt / (ms * 1e-3) / 1e12,
                     "frac": byt / (ms * 1e-3) / 1e9 / peak, "status": int(status)}
        b.close()
        del out
    print(json.dumps({"metric": "batched bulk-copy runner by pool class: algorithmic bytes per second",
                      "peak_gbs": peak, "peak_kind": kind, "passes_per_launch": passes, "runs": runs,
                      "tuning": [0, 2560, 2048], "classes": res}), flush=True)


def serve_bench(n_clients: int = 10_000, n_requests: int = 20_000, rate: float = 50_000.0,
                budget_gb: float = 40.0, passes_per_tick: int = 2, ctas_per_sm: int = 0,
                cpu_baseline: bool = True, tick=None, parity: bool = True) -> dict:
    """Serving loop: n_clients generators (n = 4, N log-uniform on
    [2^10, 2^20], frac = 1/3), Poisson arrivals at `rate`, counts log-uniform
    on [2^10, 2^24], mu ~ U[-10, 10], sigma ~ U[0.1, 10], admitted against a
    device-memory budget; p50/p99 latency and sustained variates/s."""
    import numpy as np
    import torch
    from paper_1004_3114_gb300 import wallace as W
    from paper_1004_3114_gb300.workloads import serving_clients, serving_requests
    Ns = serving_clients(n_clients)
    seeds = np.arange(n_clients, dtype=np.uint32) + 20000
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    srv = W.Server(4, Ns, seeds, 1 / 3, int(budget_gb * (1 << 30)), stream=stream)
    create_s = time.perf_counter() - t0
    # pools of up to 24576 values stay in shared memory (the bulk-copy
    # runner's block holds them; 8192 with the 256-thread kernel only)
    srv.set_tuning(passes_per_tick, 24576 if ctas_per_sm == 0 else 4096, ctas_per_sm)
    if tick:
        srv.set_tick(*tick)
    tr = serving_requests(n_requests, n_clients, rate)
    t0 = time.perf_counter()
    lat = srv.run_trace(tr["arrival_s"], tr["client"], tr["count"], tr["mu"], tr["sigma"])
    wall = time.perf_counter() - t0
    st = srv.stats()
    values = int(tr["count"].sum())
    peak, kind = hbm_peak()
    bytes_moved = 28 * values        # per returned value at f = 3: 3 x 8 B pool read+write + 4 B out
    parity = serve_sampled_parity(srv, Ns, seeds, tr) if parity else None
    srv.close()
    cpu = serve_cpu_baseline(Ns, seeds, tr) if cpu_baseline else None
    offered = values / float(tr["arrival_s"][-1])
    return {
        "metric": "served N(mu, sigma^2) variates/s", "value": values / st.elapsed_s, "unit": UNIT,
        "cpu_baseline": cpu,
        "workload": f"{n_clients} clients, n=4, N log-uniform on [2^10, 2^20], frac=1/3; "
                    f"{n_requests} requests, Poisson {rate:.0f}/s, count log-uniform on [2^10, 2^24], "
                    f"mu~U[-10,10], sigma~U[0.1,10]; budget {budget_gb} GB",
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "values": values, "elapsed_s": st.elapsed_s, "wall_s": wall,
        "offered_values_per_s": offered, "served_over_offered": values / st.elapsed_s / offered,
        "ticks": int(st.ticks), "hbm_peak_gb": st.hbm_peak / 2**30, "hbm_budget_gb": st.hbm_budget / 2**30,
        "host_tick_s": st.host_tick_s, "host_wait_s": st.host_wait_s, "items": int(st.items),
        "mean_admit_wait_ms": st.mean_admit_wait_ms,
        "roofline": {"bound": "hbm", "achieved": bytes_moved / st.elapsed_s / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": bytes_moved / st.elapsed_s / 1e9 / peak, "peak_kind": kind,
                     "bytes_per_value": 28},
        "passes_per_tick": passes_per_tick, "ctas_per_sm": ctas_per_sm, "tick": tick,
        "runner": "bulk-copy for one-CTA requests on 4096 <= N (n=4)" if ctas_per_sm == 0
                  else "async-copy", "create_s": create_s, "sampled_parity": parity,
        "status": int(st.status)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=15000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-passes", type=int, default=50)
    ap.add_argument("--reference-budget-s", type=float, default=90.0,
                    help="--impl reference: time budget of the timed oracle steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-stats", action="store_true",
                    help="skip the moment / KS summary of the first 10^8 draws")
    ap.add_argument("--batched", action="store_true",
                    help="4096 uneven generators in one persistent launch vs one handle each")
    ap.add_argument("--pow2", action="store_true", help="with --batched: power-of-two pool sizes")
    ap.add_argument("--batched-count", type=int, default=4096, help="with --batched: generators")
    ap.add_argument("--batched-runs", type=int, default=10, help="with --batched: timed runs of 10 passes")
    ap.add_argument("--variants-steps", type=int, default=2000, help="with --variants: passes per case")
    ap.add_argument("--variants", action="store_true",
                    help="RANN4 (n=2), per-pass sign patterns, Wilson-Hilferty and restarts on the default pool size")
    ap.add_argument("--boxmuller", action="store_true",
                    help="the Box-Muller comparison generator beside the Wallace pass")
    ap.add_argument("--small", action="store_true",
                    help="the small correctness configuration (n=4, N=256, frac=1, 1000 passes per fill)")
    ap.add_argument("--serve", action="store_true",
                    help="continuous-batching serving loop (10^4 clients, Poisson arrivals)")
    ap.add_argument("--serve-requests", type=int, default=20_000)
    ap.add_argument("--serve-rate", type=float, default=50_000.0)
    ap.add_argument("--serve-ppt", type=int, default=2)
    ap.add_argument("--serve-tick", default=None,
                    help="with --serve: semicolon-separated one_cta_max:values_per_tick settings to sweep")
    ap.add_argument("--serve-ctas", type=int, default=0,
                    help="CTAs per SM of the one-CTA requests; 0: bulk-copy runner where it applies")
    ap.add_argument("--batched-classes", action="store_true",
                    help="the bulk-copy batched runner on one class of pool sizes (lane count) at a time")
    ap.add_argument("--class", dest="classes", action="append", choices=list(BATCH_CLASSES),
                    help="with --batched-classes: only this class (repeatable)")
    ap.add_argument("--class-pools", type=int, default=1024)
    ap.add_argument("--class-passes", type=int, default=10)
    ap.add_argument("--class-runs", type=int, default=3)
    ap.add_argument("--l2", action="store_true",
                    help="multi-pass L2 kernel against one launch per pass, N = 2^14..2^22")
    ap.add_argument("--l2-grids", default="0",
                    help="with --l2: comma-separated grid sizes (0: two CTAs per SM)")
    ap.add_argument("--l2-n", type=int, default=4, help="with --l2: sub-vectors (4 or 8)")
    ap.add_argument("--l2-sizes", default="14-21",
                    help="with --l2: log2 of nu / 4, a range a-b or a comma-separated list")
    ap.add_argument("--n8", action="store_true",
                    help="n = 8 pass alone (A = J/4 - I, seed 7, frac = 1/2)")
    ap.add_argument("--n8-log2N", type=int, default=23, help="with --n8: N = 2^k")
    ap.add_argument("--n8-variant", default="auto", choices=["auto", "tiled_tma", "tiled_cluster", "twophase"],
                    help="with --n8: pass kernel")
    ap.add_argument("--n8-steps", type=int, default=2000, help="with --n8: timed passes")
    ap.add_argument("--n8-no-parity", action="store_true", help="with --n8: skip the first-pass oracle check")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line only: skip the batched, serving, n = 8 and precision objects")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON-lines file caching the batched autotuner's choice (default: tune every run)")
    ap.add_argument("--precision-study", action="store_true",
                    help="binary32 vs binary64 pool study (N=2^22, n=4 and 8, 1000 passes) instead of the benchmark")
    args = ap.parse_args()
    if args.precision_study:
        print(json.dumps(precision_study()), flush=True)
        return
    if args.l2:
        grids = tuple(int(v) for v in args.l2_grids.split(","))
        if "-" in args.l2_sizes:
            lo, hi = (int(v) for v in args.l2_sizes.split("-"))
            sizes = range(lo, hi + 1)
        else:
            sizes = [int(v) for v in args.l2_sizes.split(",")]
        print(json.dumps(l2_bench(log2_sizes=sizes, grids=grids, n=args.l2_n)), flush=True)
        return
    if args.batched:
        print(json.dumps(batched_bench(power_of_two=args.pow2, count=args.batched_count,
                                       runs=args.batched_runs, tune_cache=args.tune_cache)), flush=True)
        return
    if args.batched_classes:
        batched_classes_bench(args.classes, pools=args.class_pools, passes=args.class_passes,
                              runs=args.class_runs)
        return
    if args.small:
        small_config_bench()
        return
    if args.boxmuller:
        boxmuller_bench()
        return
    if args.variants:
        variant_bench(steps=args.variants_steps)
        return
    if args.n8:
        from paper_1004_3114_gb300 import wallace as W
        var = {"auto": W.VARIANT_AUTO, "tiled_tma": W.VARIANT_TILED_TMA,
               "tiled_cluster": W.VARIANT_TILED_CLUSTER, "twophase": W.VARIANT_TWOPHASE}[args.n8_variant]
        print(json.dumps(n8_bench(steps=args.n8_steps, N=1 << args.n8_log2N, variant=var,
                                  parity=not args.n8_no_parity)), flush=True)
        return
    if args.serve:
        ticks = [None] if not args.serve_tick else [
            tuple(int(v) for v in t.split(":")) for t in args.serve_tick.split(";")]
        for tk in ticks:
            print(json.dumps(serve_bench(n_requests=args.serve_requests, rate=args.serve_rate,
                                         passes_per_tick=args.serve_ppt, ctas_per_sm=args.serve_ctas,
                                         tick=tk, cpu_baseline=len(ticks) == 1, parity=len(ticks) == 1)),
                  flush=True)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
