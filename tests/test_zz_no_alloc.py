"""oph_build_sketches_static, the sketch entry point that allocates no device
memory, gives the same sketches as oph_build_sketches.

It exists for callers that may not allocate device memory during a call (a
serving loop on a fixed budget owned by its own pool allocator, or a
latency-critical path that cannot absorb the synchronisation a cudaMalloc /
cudaFree may bring).  Its work list lives in a fixed device array shared by
all calls, so the test makes two calls in a row with different inputs and
checks each one; it also checks the size limit.  This file is collected
last so a run that stops at the first failure has already run every other
test.
"""
import numpy as np
import pytest

from gpu_helpers import device, planes_to_rows, to_dev, torch  # noqa: F401
from paper_1805_11254_gb300 import hoph, synth

pytestmark = pytest.mark.gpu


def _inputs(n_sets, seed, D):
    sizes = synth.lognormal_sizes(n_sets, 80, 1.0, 1, 5000, seed)
    off = synth.offsets_from_sizes(sizes)
    ids = synth.counter_ids(seed, 0, int(off[-1]), D)
    return ids, off


@pytest.mark.parametrize("ab,kg", [((0, 0), 64), ((1, 2), 64)])
def test_static_entry_point_matches_allocating_one(ab, kg):
    dev = device()
    D, k = 1 << 20, 256
    with hoph.Plan(D, k, kg, *ab, seed=1) as plan:
        # calls in a row through the C ABI, different sizes and contents, each
        # smaller batch after a larger one (the shared array keeps the last
        # call's contents): two-launch sizes (60,000 and 20,011 sets), a
        # one-launch size with a multi-warp work list (9,000), the one-CTA
        # work-list kernel (3,000) and a batch too small for a work list (37)
        for n_sets, seed in ((60000, 31), (9000, 35), (20011, 32), (3000, 34), (37, 33)):
            ids, off = _inputs(n_sets, seed, D)
            d_ids, d_off = to_dev(ids, dev), to_dev(off, dev)
            want = torch.full((plan.G, n_sets, kg), -7, dtype=torch.int32, device=dev)
            got = torch.full((plan.G, n_sets, kg), -7, dtype=torch.int32, device=dev)
            hoph.oph_build_sketches(plan.handle, d_ids, d_off, n_sets, want)
            hoph.oph_build_sketches_static(plan.handle, d_ids, d_off, n_sets, got)
            assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_OK
            assert np.array_equal(planes_to_rows(got), planes_to_rows(want))


def test_static_entry_point_rejects_oversized_input():
    dev = device()
    with hoph.Plan(1 << 16, 128, 32, seed=1) as plan:
        ids, off = _inputs(10, 5, 1 << 16)
        planes = torch.empty((plan.G, 10, 32), dtype=torch.int32, device=dev)
        with pytest.raises(hoph.HophError) as e:
            hoph.oph_build_sketches_static(plan.handle, to_dev(ids, dev), to_dev(off, dev),
                                           (1 << 18) + 1, planes)
        assert e.value.code == hoph.HOPH_ERR_TOO_LARGE
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_OK
