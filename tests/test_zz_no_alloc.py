"""wallace_pass_static, the pass that allocates nothing.

It serves callers that cannot allocate device memory (for example a plug-in
whose host application owns every device buffer and forbids cudaMalloc): the
caller keeps the pool and the per-pass parameters, and the pass's scratch
lives in a fixed array inside the library.  Its results must equal, bit for
bit (the tolerance of the other parity tests), both the oracle's pass with the
same parameters and the handle API's, on two calls in a row.  This file is
collected last on purpose: a run that stops at the first failure has already
run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1004_3114_gb300 import wallace as W  # noqa: E402


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("n,N,frac", [(4, 1 << 16, 0.5), (8, 3001, 1.0), (4, 20005, 1 / 3)])
def test_static_pass_matches_oracle_two_calls(orc, n, N, frac):
    """Passes 1 and 2 of an oracle generator, the static call given the
    oracle's own strides, offsets and scale."""
    o = orc.Generator(n, N, 17, frac)
    R = o.stats().R
    pool = torch.from_numpy(o.pool32()).cuda()     # caller-held pool, rows of N
    c32 = o.stats().c32                            # scale of pass 1, from the initial pool
    out = torch.empty(R, dtype=torch.float32, device="cuda")
    for call in range(2):
        ref_out = o.fill(R, -0.75, 3.0)             # the oracle's next pass, its returned values
        st = o.stats()
        rc, res = W.pass_static(n, N, pool, st.alpha[:n], st.gamma[:n], c32, out, R, -0.75, 3.0)
        assert rc == 0 and res.status == 0 and res.bad == 0, (call, rc)
        assert np.array_equal(_bits(pool.cpu().numpy()), _bits(o.pool32())), call
        assert np.array_equal(_bits(out.cpu().numpy()), _bits(ref_out)), call
        assert res.Q == st.Q and res.q == st.q and res.S == st.S, call
        assert res.c == st.c and res.c32 == st.c32, call
        c32 = res.c32


@pytest.mark.parametrize("n,N,frac", [(4, 1 << 16, 0.5), (8, 3001, 1.0)])
def test_static_pass_matches_handle_two_calls(n, N, frac):
    h = W.Wallace(n, N, 13, frac)
    R = h.R
    out_h = torch.empty(R, dtype=torch.float32, device="cuda")
    h.fill(out_h)                                   # pass 1 through the handle
    pool = torch.from_numpy(h.pool()).cuda()        # caller-held pool, rows of N
    c32 = h.stats().c32                             # scale for pass 2
    out_s = torch.empty(R, dtype=torch.float32, device="cuda")
    for call in range(2):                           # passes 2 and 3, two calls in a row
        h.fill(out_h, 0.25, 1.5)
        st = h.stats()
        rc, res = W.pass_static(n, N, pool, st.alpha[:n], st.gamma[:n], c32, out_s, R, 0.25, 1.5)
        assert rc == 0 and res.status == 0, (call, rc)
        assert np.array_equal(_bits(pool.cpu().numpy()), _bits(h.pool())), call
        assert np.array_equal(_bits(out_s.cpu().numpy()), _bits(out_h.cpu().numpy())), call
        assert res.Q == st.Q and res.S == st.S and res.c == st.c and res.c32 == st.c32, call
        c32 = res.c32
    h.close()


def test_static_pass_rejects_pools_beyond_its_array():
    n, N = 4, W.STATIC_MAX_VALUES // 4 + 1
    pool = torch.empty(1, dtype=torch.float32, device="cuda")
    rc, _ = W.pass_static(n, N, pool, [3, 7, 15, 35], [0, 0, 0, 0], 1.0)
    assert rc == W.EINVAL


def test_static_pass_withholds_the_last_value():
    """out_count = n*N would return the value that sets the next pass's scale
    (Section 4): rejected before any work, the pool untouched."""
    n, N = 4, 1024
    pool = torch.randn(n * N, device="cuda")
    before = pool.clone()
    out = torch.empty(n * N, device="cuda")
    rc, _ = W.pass_static(n, N, pool, [3, 5, 9, 45], [1, 2, 3, 4], 1.0, out, n * N)
    assert rc == W.EINVAL
    assert torch.equal(pool, before)
    with pytest.raises(ValueError):
        W.pass_static(n, N, pool, [3, 5, 9, 45], [1, 2, 3, 4], 1.0, pool[:10], 10)   # aliases the pool
    with pytest.raises(ValueError):
        W.pass_static(n, N, pool[: n * N - 1], [3, 5, 9, 45], [1, 2, 3, 4], 1.0)     # too small
