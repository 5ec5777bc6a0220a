"""Host-side admission rules of the continuous-batching service (no GPU)."""
import numpy as np

from paper_1805_11254_gb300 import serve
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


class _FakeExecutor:
    """The executor's interface on the host: `n` lanes, each batch takes
    `service` seconds of the fake clock; a batch's requests get one pair per
    query set (the set's own index), so results can be checked per request."""

    def __init__(self, clock, n=2, service=0.004):
        self.lanes = [dict(busy=None) for _ in range(n)]
        self.clock, self.service, self.launched = clock, service, []

    def free_lane(self):
        return next((ln for ln in self.lanes if ln["busy"] is None), None)

    def launch(self, lane, reqs, bucket):
        self.launched.append((len(reqs), bucket))
        lane["busy"] = (reqs, self.clock() + self.service)

    def poll(self, now_fn, block=False):
        done = []
        for ln in self.lanes:
            if ln["busy"] is not None and self.clock() >= ln["busy"][1]:
                for r in ln["busy"][0]:
                    r.pairs = [(j, 0, 1, 0) for j in range(len(r.sets))]
                    r.done = now_fn()
                    done.append(r)
                ln["busy"] = None
        return done


def test_serve_loop_completes_every_request_once_with_its_own_results():
    """serve() over a fake clock and executor: every admitted request
    completes exactly once, after its arrival, with results for each of its
    own sets; oversized requests come back rejected; batches never exceed
    the largest bucket, and at most `n` are in flight."""
    t = [0.0]

    def clock():
        t[0] += 1e-4  # each look at the clock advances it
        return t[0]

    rng = np.random.default_rng(3)
    reqs = [serve.Request(i, [np.arange(int(rng.integers(1, 50)), dtype=np.uint32)
                              for _ in range(int(rng.integers(1, 40)))], 0.002 * i)
            for i in range(60)]
    reqs.append(serve.Request(60, [np.arange(5, dtype=np.uint32)] * 300, 0.05))  # > 256 sets
    ex = _FakeExecutor(clock)
    done = serve.serve(ex, serve.Batcher((16, 64, 256), 1 << 20), reqs, clock=clock)
    assert sorted(r.rid for r in done) == list(range(61))
    rejected = [r for r in done if r.error is not None]
    assert [r.rid for r in rejected] == [60]
    for r in done:
        if r.error is None:
            assert r.done is not None and r.done >= r.arrival
            assert r.pairs == [(j, 0, 1, 0) for j in range(len(r.sets))]
    assert all(bucket <= 256 and n >= 1 for n, bucket in ex.launched)


def test_latency_summary_and_poisson_arrivals():
    reqs = serve.poisson_requests(5000.0, 0.5, 7, lambda rng, n: [np.zeros(3, np.uint32)] * n)
    assert reqs and all(a.arrival < b.arrival for a, b in zip(reqs, reqs[1:]))
    sets = sum(len(r.sets) for r in reqs)
    assert 1500 < sets < 3500  # 5,000 sets/s for 0.5 s
    for i, r in enumerate(reqs):
        r.done = r.arrival + 0.001 * (1 + i % 10)
    s = serve.latency_summary(reqs)
    assert s["requests"] == len(reqs)
    assert 1.0 <= s["p50_ms"] <= 10.0 and s["p99_ms"] <= 10.0 + 1e-9


def test_id_capacity_follows_the_free_device_memory():
    """The executor sizes each lane's ID buffer from the free HBM it reads at
    start (a fake reader here): a reserve fraction kept back, the rest split
    over the lanes at 4 bytes per ID, capped; nothing left admits nothing."""
    free = {"bytes": 80 << 30}
    reader = lambda: free["bytes"]  # noqa: E731
    cap = serve.id_capacity_from_free_memory(reader(), 4, reserve_frac=0.25, max_ids=1 << 40)
    assert cap == (int((80 << 30) * 0.75) // 4) // 4
    assert serve.id_capacity_from_free_memory(reader(), 4, 0.25, max_ids=1 << 20) == 1 << 20
    free["bytes"] = 4 * 1000 * 2  # two lanes, no reserve: 1,000 IDs each
    assert serve.id_capacity_from_free_memory(reader(), 2, 0.0) == 1000
    free["bytes"] = 0
    assert serve.id_capacity_from_free_memory(reader(), 2, 0.25) == 0
    import pytest
    with pytest.raises(ValueError):
        serve.id_capacity_from_free_memory(1 << 30, 0)
    with pytest.raises(ValueError):
        serve.id_capacity_from_free_memory(1 << 30, 2, reserve_frac=1.0)


def test_admission_is_bounded_by_the_memory_budget():
    """With the ID capacity a small device leaves (fake reader: 2,400 bytes
    free, 2 lanes, no reserve -> 300 IDs per batch), requests are batched
    only while their IDs fit, and a request that alone exceeds it is
    rejected rather than queued; a larger device admits them together."""
    small = serve.id_capacity_from_free_memory(2400, 2, reserve_frac=0.0)
    assert small == 300
    reqs = [_req(0, [100, 100], 0.0), _req(1, [150], 0.0), _req(2, [50], 0.0),
            _req(3, [400], 0.0)]
    b = Batcher((4, 8), id_capacity=small)
    assert [b.offer(r) for r in reqs] == [True, True, True, False]
    assert [r.rid for r in b.rejected] == [3]
    got, _ = b.next_batch(0.0)
    assert [r.rid for r in got] == [0]          # 200 IDs; +150 would exceed 300
    got, _ = b.next_batch(0.0)
    assert [r.rid for r in got] == [1, 2]       # 150 + 50
    big = serve.id_capacity_from_free_memory(1 << 20, 2, reserve_frac=0.0)
    b = Batcher((4, 8), id_capacity=big)
    for r in reqs:
        r.error = None
        assert b.offer(r)
    got, bucket = b.next_batch(0.0)
    assert [r.rid for r in got] == [0, 1, 2, 3] and bucket == 8
