"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/wallace.h declares."""
import ctypes
import os

import pytest


@pytest.fixture(scope="module")
def libpath():
    from paper_1004_3114_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(libpath):
    from paper_1004_3114_gb300 import wallace as W
    names = W.header_functions()
    assert len(names) >= 18
    lib = ctypes.CDLL(libpath)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_core_entry_points_declared(libpath):
    from paper_1004_3114_gb300 import wallace as W
    names = set(W.header_functions())
    for n in ("wallace_create", "wallace_pass", "wallace_fill", "wallace_destroy"):
        assert n in names


def test_strerror_and_argument_checks_need_no_gpu(libpath):
    from paper_1004_3114_gb300 import wallace as W
    lib = W.lib()
    assert lib.wallace_strerror(0) == b"ok"
    assert b"sum-of-squares" in lib.wallace_strerror(W.ECORRUPT)
    h = ctypes.c_void_p()
    # argument validation happens before any CUDA call
    assert lib.wallace_create(3, 256, 1, 1.0, ctypes.byref(h)) == W.EINVAL
    assert lib.wallace_create(4, 2, 1, 1.0, ctypes.byref(h)) == W.EINVAL
    assert lib.wallace_create(4, 256, 1, 0.0, ctypes.byref(h)) == W.EINVAL
    assert lib.wallace_create(4, 256, 1, 1.5, ctypes.byref(h)) == W.EINVAL
    assert lib.wallace_create(4, 1 << 29, 1, 1.0, ctypes.byref(h)) == W.EINVAL
    assert lib.wallace_pass(None) == W.EINVAL
    lib.wallace_destroy(None)


def test_product_has_no_oracle_dependency():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1004_3114_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower() or f == "__init__.py", f


def test_static_pass_binding_checks_tensors_before_the_call(libpath):
    """The C entry point cannot see a tensor's size or device, so the binding
    rejects a CPU, wrongly typed or undersized pool before calling it."""
    torch = pytest.importorskip("torch")
    from paper_1004_3114_gb300 import wallace as W
    n, N = 4, 256
    for bad in (torch.zeros(n * N), torch.zeros(n * N, dtype=torch.float64)):
        with pytest.raises(ValueError):
            W.pass_static(n, N, bad, [3, 5, 9, 45], [0, 0, 0, 0], 1.0)
    with pytest.raises(ValueError):
        W.pass_static(n, N, torch.zeros(n * N), [3, 5, 9], [0, 0, 0], 1.0)   # too few strides
