"""The device-side timeout path (failure detection without a GPU fault).

Every wait inside the library's kernels is bounded: a wait that runs out sets
an error bit in the handle's device state, and the next synchronising call
returns MBO_ERR_DEVICE_TIMEOUT.  mbo_selftest_wait_timeout makes such a wait
run out on purpose -- one block waits on an mbarrier phase that nothing
completes, for about a millisecond -- and the handle must report the timeout
and then work normally.  Nothing faults, traps or hangs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1711_01365_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_1711_01365_gb300 import build
    build.build()
    from paper_1711_01365_gb300 import mbo
    return mbo


def test_bounded_wait_runs_out_and_the_handle_recovers(M):
    dims, n = (64, 1024), 3
    tau = 3.0 / 1024 ** 2
    h = M.Mbo(dims, n, tau, "f32")
    assert M.mbo_selftest_wait_timeout(h.h, 2_000_000) == 6  # MBO_ERR_DEVICE_TIMEOUT
    assert "bounded device wait" in M.mbo_last_error(h.h)
    # the error bit was cleared: a step runs and reports normally
    A = torch.tensor(O.project(I.gaussian(dims, n, 3), n), dtype=torch.float32, device="cuda")
    rec = h.step(A, want_stats=True)
    assert rec["nonfinite"] == 0 and np.isfinite(rec["energy"])
    # and a second self-test reports the timeout again
    assert M.mbo_selftest_wait_timeout(h.h, 2_000_000) == 6
    h.close()
