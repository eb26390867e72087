"""ctypes access to the plain-C oracle of Wallace's generator (Brent, RANN4).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark.  The product library never imports it.

`build()` compiles `wallace_oracle.c` with gcc (strict IEEE: no FMA
contraction, no fast-math) into `liborc.so` next to this file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "wallace_oracle.c")
HDR = os.path.join(HERE, "wallace_oracle.h")
LIB = os.path.join(HERE, "liborc.so")

FP32, FP64 = 0, 1
CHI_WH = 0x100   # mode flag: Wilson-Hilferty chi-squared sample
SIGNS = 0x200    # mode flag: random sign pattern per pass (matrix A D_k)
OK, EINVAL, ENOMEM, ECORRUPT = 0, 1, 2, 4

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
          "-fno-fast-math", "-fexcess-precision=standard", "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or older than its sources."""
    stale = (not os.path.exists(LIB)
             or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


class Stats(C.Structure):
    _fields_ = [
        ("q_lo", C.c_uint64), ("q_hi", C.c_uint64), ("q", C.c_double),
        ("S", C.c_double), ("c", C.c_double), ("c32", C.c_float),
        ("drift", C.c_double), ("passes", C.c_int64), ("status", C.c_int),
        ("bad", C.c_int), ("lcg", C.c_uint64), ("alpha", C.c_int32 * 8),
        ("gamma", C.c_int64 * 8), ("R", C.c_int64), ("cursor", C.c_int64),
        ("signs", C.c_uint32), ("rot_c", C.c_double), ("rot_s", C.c_double),
    ]

    @property
    def Q(self) -> int:
        return (int(self.q_hi) << 64) | int(self.q_lo)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        sig = {
            "orc_splitmix64": (C.c_uint64, [C.c_uint64]),
            "orc_seed_state": (C.c_uint64, [C.c_uint32, C.c_uint32]),
            "orc_lcg_next": (C.c_uint32, [C.POINTER(C.c_uint64)]),
            "orc_log_w": (C.c_double, [C.c_uint64]),
            "orc_sincos_quarter": (None, [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "orc_sincos_2pi": (None, [C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "orc_box_muller": (None, [C.c_uint32, C.c_uint32, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
            "orc_lcg_jump": (C.c_uint64, [C.c_uint64, C.c_uint64]),
            "orc_draw_rotation": (None, [C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "orc_pass_rot32": (None, [C.c_int64, f32p, f32p, i32p, i64p, C.c_float, C.c_float]),
            "orc_pass_rot64": (None, [C.c_int64, f64p, f64p, i32p, i64p, C.c_double, C.c_double]),
            "orc_set_restart": (None, [C.c_void_p, C.c_int64]),
            "orc_restart_pool": (None, [C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, f32p]),
            "orc_boxmuller_stream": (None, [C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, C.c_float,
                                            C.c_float, f32p]),
            "orc_stride_candidates": (C.c_int, [C.c_int, C.c_int64, i32p]),
            "orc_draw_params": (None, [C.c_int, C.c_int64, C.POINTER(C.c_uint64), i32p, i64p]),
            "orc_transform32": (None, [C.c_int, f32p, C.c_float, f32p]),
            "orc_transform64": (None, [C.c_int, f64p, C.c_double, f64p]),
            "orc_term32": (C.c_uint64, [C.c_float, C.POINTER(C.c_int)]),
            "orc_pass_explicit32": (None, [C.c_int, C.c_int64, f32p, f32p, i32p, i64p, C.c_float,
                                           C.c_uint32]),
            "orc_pass_explicit64": (None, [C.c_int, C.c_int64, f64p, f64p, i32p, i64p, C.c_double,
                                           C.c_uint32]),
            "orc_sumsq32": (C.c_int, [f32p, C.c_int64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
            "orc_sumsq64": (C.c_int, [f64p, C.c_int64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
            "orc_returned_count": (C.c_int64, [C.c_int64, C.c_double]),
            "orc_create": (C.c_void_p, [C.c_int, C.c_int64, C.c_uint32, C.c_uint32, C.c_double, C.c_int]),
            "orc_pass": (C.c_int, [C.c_void_p]),
            "orc_fill32": (C.c_int, [C.c_void_p, f32p, C.c_int64, C.c_float, C.c_float]),
            "orc_fill64": (C.c_int, [C.c_void_p, f64p, C.c_int64, C.c_double, C.c_double]),
            "orc_get_pool32": (None, [C.c_void_p, f32p]),
            "orc_get_pool64": (None, [C.c_void_p, f64p]),
            "orc_get_stats": (None, [C.c_void_p, C.POINTER(Stats)]),
            "orc_set_pool32": (None, [C.c_void_p, f32p]),
            "orc_destroy": (None, [C.c_void_p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ---- thin helpers over the building blocks --------------------------------

def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(x))


def seed_state(seed: int, stream: int = 0) -> int:
    return int(lib().orc_seed_state(seed, stream))


def lcg_stream(state: int, count: int) -> tuple[np.ndarray, int]:
    """`count` uniforms from the given state; returns (uniforms, new state)."""
    s = C.c_uint64(state)
    out = np.empty(count, dtype=np.uint32)
    f = lib().orc_lcg_next
    for k in range(count):
        out[k] = f(C.byref(s))
    return out, int(s.value)


def log_w(w: int) -> float:
    return float(lib().orc_log_w(w))


def sincos_quarter(g: float) -> tuple[float, float]:
    s, c = C.c_double(), C.c_double()
    lib().orc_sincos_quarter(g, C.byref(s), C.byref(c))
    return s.value, c.value


def sincos_2pi(u: int) -> tuple[float, float]:
    s, c = C.c_double(), C.c_double()
    lib().orc_sincos_2pi(u, C.byref(s), C.byref(c))
    return s.value, c.value


def box_muller(u1: int, u2: int) -> tuple[np.float32, np.float32]:
    a, b = C.c_float(), C.c_float()
    lib().orc_box_muller(u1, u2, C.byref(a), C.byref(b))
    return np.float32(a.value), np.float32(b.value)


def boxmuller_stream(seed: int, stream: int, offset: int, count: int, mu: float = 0.0,
                     sigma: float = 1.0) -> np.ndarray:
    out = np.empty(count, dtype=np.float32)
    lib().orc_boxmuller_stream(seed, stream, offset, count, np.float32(mu), np.float32(sigma), out)
    return out


def stride_candidates(n: int, N: int) -> list[int]:
    """Candidate strides of a pass for n = 4 or 8 (Sections 3 and 7), increasing."""
    cand = np.zeros(11, dtype=np.int32)
    k = lib().orc_stride_candidates(n, N, cand)
    return [int(v) for v in cand[:k]]


def draw_params(n: int, N: int, state: int) -> tuple[np.ndarray, np.ndarray, int]:
    s = C.c_uint64(state)
    alpha = np.zeros(8, dtype=np.int32)
    gamma = np.zeros(8, dtype=np.int64)
    lib().orc_draw_params(n, N, C.byref(s), alpha, gamma)
    return alpha[:n].copy(), gamma[:n].copy(), int(s.value)


def transform32(g: np.ndarray, c: float) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.float32)
    y = np.empty_like(g)
    lib().orc_transform32(len(g), g, np.float32(c), y)
    return y


def transform64(g: np.ndarray, c: float) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.float64)
    y = np.empty_like(g)
    lib().orc_transform64(len(g), g, float(c), y)
    return y


def term32(y: float) -> tuple[int, int]:
    bad = C.c_int(0)
    t = int(lib().orc_term32(np.float32(y), C.byref(bad)))
    return t, bad.value


def _pad8(a, dtype):
    out = np.zeros(8, dtype=dtype)
    out[:len(a)] = a
    return out


def pass_explicit32(n, N, x, alpha, gamma, c, signs: int = 0) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().orc_pass_explicit32(n, N, x, y, _pad8(alpha, np.int32), _pad8(gamma, np.int64), np.float32(c),
                              signs)
    return y


def pass_explicit64(n, N, x, alpha, gamma, c, signs: int = 0) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().orc_pass_explicit64(n, N, x, y, _pad8(alpha, np.int32), _pad8(gamma, np.int64), float(c),
                              signs)
    return y


def sumsq32(pool) -> tuple[int, int]:
    pool = np.ascontiguousarray(pool, dtype=np.float32)
    lo, hi = C.c_uint64(), C.c_uint64()
    bad = lib().orc_sumsq32(pool, len(pool), C.byref(lo), C.byref(hi))
    return (int(hi.value) << 64) | int(lo.value), int(bad)


def sumsq64(pool) -> tuple[int, int]:
    pool = np.ascontiguousarray(pool, dtype=np.float64)
    lo, hi = C.c_uint64(), C.c_uint64()
    bad = lib().orc_sumsq64(pool, len(pool), C.byref(lo), C.byref(hi))
    return (int(hi.value) << 64) | int(lo.value), int(bad)


def returned_count(nu: int, frac: float) -> int:
    return int(lib().orc_returned_count(nu, frac))


class Generator:
    """One oracle generator: create / pass_ / fill / pool / stats."""

    def __init__(self, n: int, N: int, seed: int, frac: float = 1.0,
                 mode: int = FP32, stream: int = 0):
        self.n, self.N, self.mode = n, N, mode & ~(CHI_WH | SIGNS)
        self.chi_wh = bool(mode & CHI_WH)
        self.nu = n * N
        self._h = lib().orc_create(n, N, seed, stream, frac, mode)
        if not self._h:
            raise ValueError(f"orc_create rejected n={n} N={N} frac={frac} mode={mode}")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_restart(self, interval: int) -> None:
        lib().orc_set_restart(self._h, interval)

    def pass_(self) -> int:
        return int(lib().orc_pass(self._h))

    def fill(self, count: int, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
        if self.mode == FP32:
            out = np.empty(count, dtype=np.float32)
            lib().orc_fill32(self._h, out, count, np.float32(mu), np.float32(sigma))
        else:
            out = np.empty(count, dtype=np.float64)
            lib().orc_fill64(self._h, out, count, float(mu), float(sigma))
        return out

    def pool32(self) -> np.ndarray:
        out = np.empty(self.nu, dtype=np.float32)
        lib().orc_get_pool32(self._h, out)
        return out

    def pool64(self) -> np.ndarray:
        out = np.empty(self.nu, dtype=np.float64)
        lib().orc_get_pool64(self._h, out)
        return out

    def set_pool32(self, pool) -> None:
        lib().orc_set_pool32(self._h, np.ascontiguousarray(pool, dtype=np.float32))

    def stats(self) -> Stats:
        st = Stats()
        lib().orc_get_stats(self._h, C.byref(st))
        return st
