"""Host-side admission rules of the continuous-batching service (no GPU)."""
import numpy as np

from paper_1805_11254_gb300.serve import Batcher, Request, pack_batch


def _req(rid, sizes, t):
    return Request(rid, [np.arange(s, dtype=np.uint32) + rid for s in sizes], t)


def test_fifo_admission_by_arrival_slots_and_ids():
    b = Batcher((4, 8), id_capacity=100)
    reqs = [_req(0, [10, 10], 0.0), _req(1, [10] * 4, 0.1), _req(2, [31, 30], 0.2),
            _req(3, [5], 5.0)]
    for r in reqs:
        assert b.offer(r)
    got, bucket = b.next_batch(0.05)         # only request 0 has arrived
    assert [r.rid for r in got] == [0] and bucket == 4
    got, bucket = b.next_batch(1.0)          # 1 fits (60 ids), 2 would exceed 100 ids
    assert [r.rid for r in got] == [1] and bucket == 4
    got, bucket = b.next_batch(1.0)
    assert [r.rid for r in got] == [2] and bucket == 4
    assert b.next_batch(1.0) == ([], 0)      # request 3 not arrived yet
    got, bucket = b.next_batch(6.0)
    assert [r.rid for r in got] == [3]


def test_batches_fill_up_to_the_largest_bucket():
    b = Batcher((2, 4, 8), id_capacity=10 ** 6)
    for i in range(5):
        b.offer(_req(i, [1, 1, 1], 0.0))
    got, bucket = b.next_batch(0.0)
    assert len(got) == 2 and bucket == 8      # 3 + 3 slots, a third request would need 9
    got, bucket = b.next_batch(0.0)
    assert len(got) == 2 and bucket == 8


def test_oversized_requests_are_rejected_not_queued():
    b = Batcher((4,), id_capacity=50)
    assert not b.offer(_req(0, [1] * 5, 0.0))
    assert not b.offer(_req(1, [60], 0.0))
    assert not b.offer(Request(2, [], 0.0))
    assert [r.rid for r in b.rejected] == [0, 1, 2] and b.pending() == 0
    assert all(r.error for r in b.rejected)


def test_pack_batch_pads_with_empty_sets():
    reqs = [_req(0, [3, 0], 0.0), _req(7, [2], 0.0)]
    h_ids = np.zeros(16, dtype=np.int32)
    h_off = np.full(9, -1, dtype=np.int64)
    n, owner = pack_batch(reqs, 8, h_ids, h_off)
    assert n == 5
    assert h_off.tolist() == [0, 3, 3, 5, 5, 5, 5, 5, 5]
    assert h_ids[:5].tolist() == [0, 1, 2, 7, 8]
    assert [(r.rid, j) for r, j in owner] == [(0, 0), (0, 1), (7, 0)]
