"""Failure detection of the device-side waits, without a GPU fault.

Every shared-memory barrier wait of the bulk-copy kernels is bounded: after
its cycle budget (about a second) the kernel records WALLACE_ETIMEOUT and
returns instead of hanging.  Here a barrier that nothing ever arrives at
makes the wait run out; the status comes back to the host, a wait on a
completed barrier still returns, and the same context then runs a pass that
matches the oracle bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_bounded_wait_gives_up_and_context_stays_usable(orc):
    from paper_1004_3114_gb300 import wallace as W
    rc, completed = W.selftest_bounded_wait()
    assert rc == W.ETIMEOUT
    assert completed
    g = W.Wallace(4, 1 << 14, 5, 0.5)
    out = torch.empty(3 * g.R, dtype=torch.float32, device="cuda")
    g.fill(out)
    assert g.sync() == 0
    o = orc.Generator(4, 1 << 14, 5, 0.5)
    ref = o.fill(3 * g.R)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    g.close()
