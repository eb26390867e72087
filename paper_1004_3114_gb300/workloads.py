"""Seeded synthetic workloads (sizes, seeds, request mixes).

Holds none of the generator's arithmetic: it only draws the shapes of the
benchmark and test workloads (pool sizes, seeds, request mixes) with numpy's
own PCG64 generator, so every consumer sees the same inputs.
"""
from __future__ import annotations

import numpy as np


def batch_sizes(count: int = 4096, lo_log2: float = 8.0, hi_log2: float = 18.0, seed: int = 4096,
                power_of_two: bool = False) -> np.ndarray:
    """Pool lengths N_s log-uniform on [2^lo, 2^hi]: floor(2^(lo + (hi-lo) u)),
    or 2^floor(lo + (hi-lo+1) u) capped at 2^hi for the power-of-two variant."""
    u = np.random.default_rng(seed).random(count)
    if power_of_two:
        e = np.minimum(np.floor(lo_log2 + (hi_log2 - lo_log2 + 1) * u), hi_log2)
        return (2 ** e).astype(np.int64)
    return np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)


def serving_clients(count: int = 10_000, lo_log2: float = 10.0, hi_log2: float = 20.0,
                    seed: int = 5000) -> np.ndarray:
    """Per-client pool lengths, log-uniform on [2^lo, 2^hi]."""
    u = np.random.default_rng(seed).random(count)
    return np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)


def serving_requests(n_requests: int, n_clients: int, rate_per_s: float = 50_000.0,
                     lo_log2: float = 10.0, hi_log2: float = 24.0, seed: int = 5001):
    """Poisson arrivals (exponential gaps at `rate_per_s`), a uniformly chosen
    client, a count log-uniform on [2^lo, 2^hi], mu ~ U[-10, 10] and
    sigma ~ U[0.1, 10] per request.  Returns a dict of numpy arrays."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    return {
        "arrival_s": np.cumsum(gaps),
        "client": rng.integers(0, n_clients, n_requests),
        "count": np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * rng.random(n_requests))).astype(np.int64),
        "mu": rng.uniform(-10.0, 10.0, n_requests).astype(np.float32),
        "sigma": rng.uniform(0.1, 10.0, n_requests).astype(np.float32),
    }
