"""Precision study at full size, end to end against the oracle.

N = 2^22, seed 3, 1000 passes, n = 4 (A = J/2 - I) and n = 8 (A = J/4 - I):
  - the binary32 pool (exact integer sum of squares, binary64 scale) against
    an independent binary32 oracle run, and the binary64-pool mode against a
    binary64 oracle run, each bit for bit: every pass's Q, S, c, drift,
    strides, offsets and uniform state, and the whole pool every 500 passes;
  - the binary32 pool's deviation from the binary64 one after 1000 passes.
    The map is an isometry, so rounding errors random-walk (about
    sqrt(3k) 2^-24 |y| RMS after k passes) and the chi-squared rescale keeps
    the scale from drifting; measured max 9.1e-6 (n = 4) and 8.9e-6 (n = 8),
    RMS 1.7e-6, so the bounds are 2e-5 max and 4e-6 RMS.
The four oracle runs start together on host threads (the oracle's C calls
release the GIL) and run while the GPU runs its passes.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1004_3114_gb300 import wallace as W  # noqa: E402

N, SEED, PASSES, POOL_EVERY = 1 << 22, 3, 1000, 500


def _scalars(st, n):
    return (st.Q, st.S, st.c, st.c32, st.drift, st.passes, st.lcg,
            tuple(st.alpha[:n]), tuple(st.gamma[:n]), st.status)


def _oracle_run(orc, n, mode):
    o = orc.Generator(n, N, SEED, 1.0, mode=mode)
    get = o.pool32 if mode == orc.FP32 else o.pool64
    per_pass, pools = [], {}
    for k in range(1, PASSES + 1):
        o.pass_()
        per_pass.append(_scalars(o.stats(), n))
        if k % POOL_EVERY == 0:
            pools[k] = get()
    o.close()
    return per_pass, pools


def _gpu_run(n, mode):
    g = W.Wallace(n, N, SEED, 1.0, mode=mode)
    get = g.pool if mode == W.FP32 else g.pool64
    per_pass, pools = [], {}
    for k in range(1, PASSES + 1):
        g.pass_()
        per_pass.append(_scalars(g.stats(), n))
        if k % POOL_EVERY == 0:
            pools[k] = get()
    assert g.sync() == 0
    g.close()
    return per_pass, pools


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


@pytest.fixture(scope="module")
def oracle_runs(orc):
    ex = ThreadPoolExecutor(4)
    futs = {(n, m): ex.submit(_oracle_run, orc, n, m) for n in (4, 8) for m in (orc.FP32, orc.FP64)}
    yield futs
    ex.shutdown(wait=True)


@pytest.mark.parametrize("n", [4, 8])
def test_precision_study_1000_passes_against_oracle(orc, oracle_runs, n):
    g32 = _gpu_run(n, W.FP32)
    g64 = _gpu_run(n, W.FP64POOL)
    o32, o64 = oracle_runs[(n, orc.FP32)].result(), oracle_runs[(n, orc.FP64)].result()
    for name, (gp, gpools), (op, opools) in (("binary32", g32, o32), ("binary64", g64, o64)):
        for k, (a, b) in enumerate(zip(gp, op)):
            assert a == b, f"{name} pool, pass {k + 1}: GPU {a} oracle {b}"
        for k in opools:
            assert np.array_equal(_bits(gpools[k]), _bits(opools[k])), f"{name} pool after {k} passes"
    # binary32 against binary64 after 1000 passes (Section 4's rescale keeps the scale)
    dev = np.abs(o32[1][PASSES].astype(np.float64) - o64[1][PASSES])
    rms = float(np.sqrt((dev ** 2).mean()))
    assert dev.max() <= 2e-5, dev.max()
    assert rms <= 4e-6, rms
    # per-pass drift q_k / S_{k-1} - 1 of the binary32 pool: rounding only
    assert max(abs(p[4]) for p in o32[0]) < 1e-6
