"""Failure detection without faulting the GPU: bounded device waits give up
and report through the status word; device-side errors and host-side
argument errors surface as status codes."""
import numpy as np
import pytest

from gpu_helpers import device, to_dev, torch  # noqa: F401
from paper_1805_11254_gb300 import hoph

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_stays_usable():
    dev = device()
    with hoph.Plan(1 << 12, 64, 16, seed=1) as plan:
        hoph.hoph_check_bounded_wait(plan.handle, 50_000_000)  # 50 ms on a barrier nobody completes
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_ERR_TIMEOUT
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_OK
        # the context still works: a sketch right after the timeout
        ids = np.arange(100, dtype=np.uint32)
        off = np.asarray([0, 100], dtype=np.int64)
        planes = plan.sketch(to_dev(ids, dev), to_dev(off, dev), 1)
        plan.check()
        assert planes.shape == (4, 1, 16)


def test_invalid_limits_and_arguments_are_rejected_on_the_host():
    device()
    with hoph.Plan(1 << 12, 64, 16, seed=1) as plan:
        for bad in (0, 3_000_000_000):
            with pytest.raises(hoph.HophError) as e:
                hoph.hoph_check_bounded_wait(plan.handle, bad)
            assert e.value.code == hoph.HOPH_ERR_PARAM
        with pytest.raises(hoph.HophError):
            hoph.hoph_query_batch(plan.handle, 99, 0, 1, 0, 1, 0, 0, 0)
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_OK
