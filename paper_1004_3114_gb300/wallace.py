"""Python binding of libwallace.so (include/wallace.h), names as in the C ABI.

Argument marshalling only: every step of the generator runs in the library's
CUDA kernels.  Device buffers are torch tensors (their data_ptr is passed),
and the handle runs on the caller's current torch CUDA stream unless another
stream is given.  Importing this module raises if the library is missing:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libwallace.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "wallace.h")

OK, EINVAL, ENOMEM, ECORRUPT, ECUDA, ETIMEOUT, ESTATE = 0, 1, 2, 4, 8, 16, 32
FP32, FP64POOL = 0, 1
CHI_WH = 0x100   # mode flag: Wilson-Hilferty chi-squared sample
MATRIX_SIGNS = 0x200   # mode flag: random sign pattern per pass (matrix A D_k)
VARIANT_AUTO, VARIANT_GATHER, VARIANT_TILED, VARIANT_FUSED = 0, 1, 2, 3
VARIANT_TILED_ASYNC, VARIANT_TILED_TMA, VARIANT_TWOPHASE, VARIANT_L2RUN = 4, 5, 6, 7
VARIANT_TILED_CLUSTER = 8

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")


class Stats(C.Structure):
    _fields_ = [
        ("q_lo", C.c_uint64), ("q_hi", C.c_uint64), ("q", C.c_double), ("S", C.c_double),
        ("c", C.c_double), ("c32", C.c_float), ("drift", C.c_double), ("passes", C.c_int64),
        ("status", C.c_int32), ("bad", C.c_int32), ("lcg", C.c_uint64),
        ("alpha", C.c_int32 * 8), ("gamma", C.c_int64 * 8), ("R", C.c_int64),
        ("cursor", C.c_int64), ("kernel_ms", C.c_double), ("kernel_launches", C.c_int64), ("launches", C.c_int64),
        ("signs", C.c_uint32), ("rot_c", C.c_double), ("rot_s", C.c_double),
    ]

    @property
    def Q(self) -> int:
        return (int(self.q_hi) << 64) | int(self.q_lo)


class ServerStats(C.Structure):
    _fields_ = [
        ("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
        ("queued", C.c_int64), ("active", C.c_int64), ("ticks", C.c_int64),
        ("values_delivered", C.c_int64), ("hbm_budget", C.c_int64), ("hbm_in_use", C.c_int64),
        ("hbm_peak", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
        ("mean_ms", C.c_double), ("elapsed_s", C.c_double), ("status", C.c_int32),
        ("pad_", C.c_int32), ("host_tick_s", C.c_double), ("host_wait_s", C.c_double),
        ("items", C.c_int64), ("mean_admit_wait_ms", C.c_double),
    ]


class PassResult(C.Structure):
    _fields_ = [
        ("q_lo", C.c_uint64), ("q_hi", C.c_uint64), ("q", C.c_double), ("S", C.c_double),
        ("c", C.c_double), ("c32", C.c_float), ("bad", C.c_int32), ("status", C.c_int32),
    ]

    @property
    def Q(self) -> int:
        return (int(self.q_hi) << 64) | int(self.q_lo)


STATIC_MAX_VALUES = 1 << 20

_lib = C.CDLL(LIB_PATH)
_h = C.c_void_p
_SIGS = {
    "wallace_create": (C.c_int, [C.c_int, C.c_int64, C.c_uint32, C.c_double, C.POINTER(_h)]),
    "wallace_create_ex": (C.c_int, [C.c_int, C.c_int64, C.c_uint32, C.c_uint32, C.c_double,
                                    C.c_int, C.c_void_p, C.POINTER(_h)]),
    "wallace_destroy": (None, [_h]),
    "wallace_pass": (C.c_int, [_h]),
    "wallace_fill": (C.c_int, [_h, C.c_void_p, C.c_int64, C.c_float, C.c_float]),
    "wallace_fill64": (C.c_int, [_h, C.c_void_p, C.c_int64, C.c_double, C.c_double]),
    "wallace_fill_host": (C.c_int, [_h, C.c_void_p, C.c_int64, C.c_float, C.c_float]),
    "wallace_set_stream": (C.c_int, [_h, C.c_void_p]),
    "wallace_set_variant": (C.c_int, [_h, C.c_int]),
    "wallace_set_timing": (C.c_int, [_h, C.c_int]),
    "wallace_set_restart": (C.c_int, [_h, C.c_int64]),
    "wallace_set_l2_grid": (C.c_int, [_h, C.c_int]),
    "wallace_sync": (C.c_int, [_h]),
    "wallace_stats": (C.c_int, [_h, C.POINTER(Stats)]),
    "wallace_get_pool": (C.c_int, [_h, C.c_void_p]),
    "wallace_get_pool64": (C.c_int, [_h, C.c_void_p]),
    "wallace_set_pool": (C.c_int, [_h, C.c_void_p]),
    "wallace_clear_error": (C.c_int, [_h]),
    "wallace_returned_per_pass": (C.c_int64, [_h]),
    "wallace_strerror": (C.c_char_p, [C.c_int]),
    "wallace_batch_create": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_void_p, C.POINTER(C.c_void_p)]),
    "wallace_batch_create_ex": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                          C.c_void_p, C.POINTER(C.c_void_p)]),
    "wallace_batch_set_restart": (C.c_int, [C.c_void_p, C.c_int64]),
    "wallace_batch_destroy": (None, [C.c_void_p]),
    "wallace_batch_run": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_float, C.c_float]),
    "wallace_batch_out_offset": (C.c_int64, [C.c_void_p, C.c_int, C.c_int64]),
    "wallace_batch_returned_per_pass": (C.c_int64, [C.c_void_p, C.c_int]),
    "wallace_batch_sync": (C.c_int, [C.c_void_p]),
    "wallace_batch_stats": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Stats)]),
    "wallace_batch_get_pool": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "wallace_batch_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int64]),
    "wallace_batch_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                           C.POINTER(C.c_int64)]),
    "wallace_batch_autotune": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int]),
    "wallace_server_create": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double,
                                        C.c_int64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "wallace_server_destroy": (None, [C.c_void_p]),
    "wallace_server_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int]),
    "wallace_server_set_tick": (C.c_int, [_h, C.c_int64, C.c_int64]),
    "wallace_server_set_restart": (C.c_int, [_h, C.c_int64]),
    "wallace_server_create_ex": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                           C.c_int64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "wallace_server_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_float, C.c_float,
                                        C.POINTER(C.c_int64)]),
    "wallace_server_progress": (C.c_int, [C.c_void_p]),
    "wallace_server_drain": (C.c_int, [C.c_void_p]),
    "wallace_server_poll": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "wallace_server_result": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "wallace_server_release": (C.c_int, [C.c_void_p, C.c_int64]),
    "wallace_server_run_trace": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "wallace_server_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "wallace_pass_static": (C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_float, C.c_void_p, C.c_int64, C.c_float, C.c_float,
                                      C.POINTER(PassResult), C.c_void_p]),
    "wallace_boxmuller_fill": (C.c_int, [C.c_uint32, C.c_uint32, C.c_int64, C.c_void_p, C.c_int64,
                                         C.c_float, C.c_float, C.c_int, C.c_void_p]),
    "wallace_selftest_bounded_wait": (C.c_int, [C.POINTER(C.c_int)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def lib() -> C.CDLL:
    return _lib


def header_functions() -> list[str]:
    """Names of the functions include/wallace.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(wallace_\w+)\s*\(", text, re.M)))


class Batch:
    """Many generators advanced in one launch (wallace_batch_*)."""

    def __init__(self, n: int, Ns, seeds, frac: float = 1.0, stream=None, mode: int = FP32):
        Ns = np.ascontiguousarray(Ns, dtype=np.int64)
        seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
        assert Ns.size == seeds.size
        self.n, self.count = n, int(Ns.size)
        self.N = Ns.copy()
        h = C.c_void_p()
        rc = _lib.wallace_batch_create_ex(self.count, n, Ns.ctypes.data, seeds.ctypes.data, frac, mode,
                                          _stream_ptr(stream), C.byref(h))
        _check(rc, "wallace_batch_create_ex")
        self._h = h
        self.R = np.array([_lib.wallace_batch_returned_per_pass(h, s) for s in range(self.count)],
                          dtype=np.int64)

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.wallace_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def out_offset(self, s: int, passes: int) -> int:
        return int(_lib.wallace_batch_out_offset(self._h, s, passes))

    def out_size(self, passes: int) -> int:
        return self.out_offset(self.count, passes)

    def run(self, passes: int, out=None, mu: float = 0.0, sigma: float = 1.0) -> int:
        ptr = C.c_void_p(out.data_ptr()) if out is not None else None
        return _check(_lib.wallace_batch_run(self._h, passes, ptr, mu, sigma), "wallace_batch_run",
                      allow=ECORRUPT)

    def set_restart(self, interval: int) -> None:
        _check(_lib.wallace_batch_set_restart(self._h, interval), "wallace_batch_set_restart")

    def sync(self) -> int:
        return _check(_lib.wallace_batch_sync(self._h), "wallace_batch_sync", allow=ECORRUPT)

    def stats(self, s: int) -> Stats:
        st = Stats()
        _check(_lib.wallace_batch_stats(self._h, s, C.byref(st)), "wallace_batch_stats",
               allow=ECORRUPT)
        return st

    def pool(self, s: int) -> np.ndarray:
        out = np.empty(self.n * int(self.N[s]), dtype=np.float32)
        _check(_lib.wallace_batch_get_pool(self._h, s, out.ctypes.data), "wallace_batch_get_pool",
               allow=ECORRUPT)
        return out

    def set_tuning(self, ctas_per_sm: int, etarget: int, fused_max: int) -> None:
        _check(_lib.wallace_batch_set_tuning(self._h, ctas_per_sm, etarget, fused_max),
               "wallace_batch_set_tuning")

    def tuning(self) -> tuple[int, int, int]:
        a, b, c = C.c_int(), C.c_int(), C.c_int64()
        _lib.wallace_batch_get_tuning(self._h, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def autotune(self, cache_path: str | None = None, trial_passes: int = 2) -> tuple[int, int, int]:
        p = cache_path.encode() if cache_path else None
        _check(_lib.wallace_batch_autotune(self._h, p, trial_passes), "wallace_batch_autotune")
        return self.tuning()


class Server:
    """Continuous-batching server over many client generators (wallace_server_*)."""

    def __init__(self, n: int, Ns, seeds, frac: float, hbm_budget_bytes: int, stream=None, mode: int = FP32):
        Ns = np.ascontiguousarray(Ns, dtype=np.int64)
        seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
        h = C.c_void_p()
        rc = _lib.wallace_server_create_ex(int(Ns.size), n, Ns.ctypes.data, seeds.ctypes.data, frac, mode,
                                           int(hbm_budget_bytes), _stream_ptr(stream), C.byref(h))
        _check(rc, "wallace_server_create_ex")
        self._h = h
        self.n, self.N = n, Ns.copy()

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.wallace_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, passes_per_tick: int, fused_max: int, ctas_per_sm: int) -> None:
        _check(_lib.wallace_server_set_tuning(self._h, passes_per_tick, fused_max, ctas_per_sm),
               "wallace_server_set_tuning")

    def set_restart(self, interval: int) -> None:
        _check(_lib.wallace_server_set_restart(self._h, interval), "wallace_server_set_restart")

    def set_tick(self, one_cta_max_values: int, values_per_tick: int) -> None:
        _check(_lib.wallace_server_set_tick(self._h, one_cta_max_values, values_per_tick),
               "wallace_server_set_tick")

    def submit(self, client: int, count: int, mu: float = 0.0, sigma: float = 1.0) -> int:
        rid = C.c_int64()
        _check(_lib.wallace_server_submit(self._h, client, count, mu, sigma, C.byref(rid)),
               "wallace_server_submit")
        return rid.value

    def progress(self) -> int:
        return _check(_lib.wallace_server_progress(self._h), "wallace_server_progress", allow=ECORRUPT)

    def drain(self) -> int:
        return _check(_lib.wallace_server_drain(self._h), "wallace_server_drain", allow=ECORRUPT)

    def poll(self, max_ids: int = 1 << 16) -> list[int]:
        ids = np.empty(max_ids, dtype=np.int64)
        n = C.c_int()
        _check(_lib.wallace_server_poll(self._h, ids.ctypes.data, max_ids, C.byref(n)),
               "wallace_server_poll", allow=ECORRUPT)
        return [int(x) for x in ids[:n.value]]

    def result(self, rid: int):
        """(device pointer, count, latency ms) of a completed request."""
        p, cnt, lat = C.c_void_p(), C.c_int64(), C.c_double()
        _check(_lib.wallace_server_result(self._h, rid, C.byref(p), C.byref(cnt), C.byref(lat)),
               "wallace_server_result")
        return p.value, cnt.value, lat.value

    def result_host(self, rid: int) -> np.ndarray:
        """Copy a completed request's values (server-owned device buffer) to the host."""
        import torch
        p, cnt, _ = self.result(rid)
        if cnt == 0:
            return np.empty(0, dtype=np.float32)
        torch.cuda.synchronize()
        return _device_floats(p, cnt).cpu().numpy().copy()

    def release(self, rid: int) -> None:
        _check(_lib.wallace_server_release(self._h, rid), "wallace_server_release")

    def run_trace(self, arrival_s, client, count, mu, sigma) -> np.ndarray:
        arrival_s = np.ascontiguousarray(arrival_s, dtype=np.float64)
        client = np.ascontiguousarray(client, dtype=np.int32)
        count = np.ascontiguousarray(count, dtype=np.int64)
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        sigma = np.ascontiguousarray(sigma, dtype=np.float32)
        lat = np.empty(arrival_s.size, dtype=np.float64)
        rc = _lib.wallace_server_run_trace(self._h, arrival_s.size, arrival_s.ctypes.data,
                                           client.ctypes.data, count.ctypes.data, mu.ctypes.data,
                                           sigma.ctypes.data, lat.ctypes.data)
        _check(rc, "wallace_server_run_trace", allow=ECORRUPT)
        return lat

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(_lib.wallace_server_stats(self._h, C.byref(st)), "wallace_server_stats")
        return st


def _device_floats(ptr: int, count: int):
    """A torch view of `count` float32 values at device address `ptr`."""
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (count,), "typestr": "<f4", "data": (ptr, False),
                                    "version": 3}
    return torch.as_tensor(_View(), device="cuda")


def _check_dev_f32(t, name: str, min_numel: int) -> None:
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.numel() < min_numel:
        raise ValueError(f"{name} holds {t.numel()} values, needs {min_numel}")


def pass_static(n: int, N: int, pool, alpha, gamma, c32: float, out=None, out_count: int | None = None,
                mu: float = 0.0, sigma: float = 1.0, stream=None) -> tuple[int, PassResult]:
    """wallace_pass_static: one pass on a caller-held pool (CUDA float32 tensor of
    n*N values, rows of N), using the library's fixed scratch array; returns
    (status, result).  out_count defaults to out.numel() (0 without `out`).
    The C call cannot see the tensors' sizes, so they are checked here; a pool
    beyond the scratch array's limit is passed through for the library to
    reject."""
    if len(alpha) < n or len(gamma) < n:
        raise ValueError(f"need {n} strides and offsets")
    if out_count is None:
        out_count = out.numel() if out is not None else 0
    if n * N <= STATIC_MAX_VALUES:
        _check_dev_f32(pool, "pool", n * N)
        if pool.numel() != n * N:
            raise ValueError(f"pool holds {pool.numel()} values, expected n*N = {n * N}")
    if out_count > 0:
        if out is None:
            raise ValueError("out_count > 0 needs an output tensor")
        _check_dev_f32(out, "out", out_count)
        if out.device != pool.device:
            raise ValueError("out and pool must be on the same device")
        p0, p1 = pool.data_ptr(), pool.data_ptr() + 4 * pool.numel()
        o0, o1 = out.data_ptr(), out.data_ptr() + 4 * out_count
        if o0 < p1 and p0 < o1:
            raise ValueError("out overlaps pool: the pass reads the pool while it writes out")
    a = (C.c_int32 * 8)(*[int(v) for v in alpha[:n]])
    g = (C.c_int64 * 8)(*[int(v) for v in gamma[:n]])
    res = PassResult()
    rc = _lib.wallace_pass_static(n, N, C.c_void_p(pool.data_ptr()), a, g, c32,
                                  C.c_void_p(out.data_ptr() if out is not None and out_count > 0 else 0),
                                  out_count, mu, sigma, C.byref(res), _stream_ptr(stream))
    return int(rc), res


def boxmuller_fill(out, seed: int, stream_id: int = 0, offset: int = 0, mu: float = 0.0,
                   sigma: float = 1.0, exact: bool = False, stream=None) -> None:
    """wallace_boxmuller_fill: values [offset, offset + out.numel()) of the
    Box-Muller stream of (seed, stream_id) into a CUDA float32 tensor."""
    _check(_lib.wallace_boxmuller_fill(seed, stream_id, offset, C.c_void_p(out.data_ptr()),
                                       out.numel(), mu, sigma, 1 if exact else 0, _stream_ptr(stream)),
           "wallace_boxmuller_fill")


def selftest_bounded_wait() -> tuple[int, bool]:
    """wallace_selftest_bounded_wait: (status of the wait on a barrier nothing
    arrives at -- ETIMEOUT when it gave up as designed --, whether the wait on
    a completed barrier returned)."""
    ok = C.c_int(0)
    rc = int(_lib.wallace_selftest_bounded_wait(C.byref(ok)))
    return rc, bool(ok.value)


class WallaceError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_lib.wallace_strerror(code).decode()} (status {code})")


def _check(rc: int, where: str, allow: int = 0) -> int:
    if rc & ~allow:
        raise WallaceError(rc, where)
    return rc


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


class Wallace:
    """One generator handle (wallace_create_ex ... wallace_destroy)."""

    def __init__(self, n: int, N: int, seed: int, frac: float = 1.0, *, stream_id: int = 0,
                 mode: int = FP32, stream=None):
        self.n, self.N, self.mode = n, N, mode & ~(CHI_WH | MATRIX_SIGNS)
        self.nu = n * N
        h = _h()
        rc = _lib.wallace_create_ex(n, N, seed, stream_id, frac, mode, _stream_ptr(stream),
                                    C.byref(h))
        _check(rc, "wallace_create_ex")
        self._h = h
        self.R = int(_lib.wallace_returned_per_pass(h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.wallace_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> int:
        return self._h.value

    def pass_(self) -> int:
        return _check(_lib.wallace_pass(self._h), "wallace_pass", allow=ECORRUPT)

    def fill(self, out, mu: float = 0.0, sigma: float = 1.0, count: int | None = None) -> int:
        """Fill a float32 (FP32 mode) or float64 (FP64POOL) CUDA tensor `out`."""
        count = out.numel() if count is None else count
        if self.mode == FP32:
            rc = _lib.wallace_fill(self._h, C.c_void_p(out.data_ptr()), count, mu, sigma)
        else:
            rc = _lib.wallace_fill64(self._h, C.c_void_p(out.data_ptr()), count, mu, sigma)
        return _check(rc, "wallace_fill", allow=ECORRUPT)

    def fill_host(self, out: np.ndarray, mu: float = 0.0, sigma: float = 1.0) -> int:
        """Fill a host float32 numpy array (or pinned torch CPU tensor)."""
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float32 and out.flags.c_contiguous
            ptr, count = out.ctypes.data, out.size
        else:
            ptr, count = out.data_ptr(), out.numel()
        rc = _lib.wallace_fill_host(self._h, C.c_void_p(ptr), count, mu, sigma)
        return _check(rc, "wallace_fill_host", allow=ECORRUPT)

    def set_stream(self, stream) -> None:
        _check(_lib.wallace_set_stream(self._h, _stream_ptr(stream)), "wallace_set_stream")

    def set_variant(self, variant: int) -> None:
        _check(_lib.wallace_set_variant(self._h, variant), "wallace_set_variant")

    def set_timing(self, on: bool) -> None:
        _check(_lib.wallace_set_timing(self._h, int(on)), "wallace_set_timing")

    def set_restart(self, interval: int) -> None:
        """Refill the pool by Box-Muller before every pass that follows a
        multiple of `interval` passes (0: never)."""
        _check(_lib.wallace_set_restart(self._h, interval), "wallace_set_restart")

    def set_l2_grid(self, grid: int = 0) -> None:
        """CTAs of VARIANT_L2RUN's launch (0: two per SM)."""
        _check(_lib.wallace_set_l2_grid(self._h, grid), "wallace_set_l2_grid")

    def sync(self) -> int:
        return _check(_lib.wallace_sync(self._h), "wallace_sync", allow=ECORRUPT)

    def stats(self) -> Stats:
        st = Stats()
        _check(_lib.wallace_stats(self._h, C.byref(st)), "wallace_stats", allow=ECORRUPT)
        return st

    def pool(self) -> np.ndarray:
        out = np.empty(self.nu, dtype=np.float32)
        _check(_lib.wallace_get_pool(self._h, out.ctypes.data), "wallace_get_pool", allow=ECORRUPT)
        return out

    def pool64(self) -> np.ndarray:
        out = np.empty(self.nu, dtype=np.float64)
        _check(_lib.wallace_get_pool64(self._h, out.ctypes.data), "wallace_get_pool64",
               allow=ECORRUPT)
        return out

    def set_pool(self, pool: np.ndarray) -> None:
        pool = np.ascontiguousarray(pool, dtype=np.float32)
        assert pool.size == self.nu
        _check(_lib.wallace_set_pool(self._h, pool.ctypes.data), "wallace_set_pool")

    def clear_error(self) -> None:
        _check(_lib.wallace_clear_error(self._h), "wallace_clear_error")
