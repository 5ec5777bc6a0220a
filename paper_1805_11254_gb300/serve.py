"""Continuous-batching near-duplicate query service over the C ABI.

Requests (each a list of query sets) arrive over time.  The batcher admits
waiting requests into the next batch while query slots and the device
memory for IDs last; that ID memory is sized from the free HBM read when
the service starts (the resident collection already allocated), minus a
reserve, split across the streams.  Each batch is padded to a fixed slot
count so its whole device work (H2D of the sets, OPH/HOPH sketching, the
HOPH query against the resident collection, D2H of the count and the first
accepted pairs) replays as one captured CUDA graph.  Several streams (two
by default) with a plan each keep that many batches in flight: the copies
and sketching of one overlap the queries of the others.
Results are scattered back per request; a request's pairs do not depend on
which other requests shared its batch (padding sets are empty and their
pairs are dropped).

The batcher is plain host logic (no GPU) so its admission rules are tested
on the CPU; the executor drives the GPU.
"""
import collections
import time

import numpy as np

from . import hoph


class Request:
    __slots__ = ("rid", "sets", "arrival", "n_ids", "done", "pairs", "error")

    def __init__(self, rid, sets, arrival):
        self.rid = rid
        self.sets = [np.ascontiguousarray(s, dtype=np.uint32) for s in sets]
        self.arrival = arrival
        self.n_ids = int(sum(len(s) for s in self.sets))
        self.done = None
        self.pairs = None
        self.error = None


class Batcher:
    """FIFO admission into batches bounded by query slots and ID capacity.

    slot_buckets: the batch sizes graphs exist for (ascending); a batch is
    padded up to the smallest bucket that holds it.  id_capacity: IDs the
    reserved device buffer holds per batch.  A request that alone exceeds
    either limit is rejected (error set) instead of blocking the queue."""

    def __init__(self, slot_buckets, id_capacity):
        self.buckets = sorted(slot_buckets)
        self.max_slots = self.buckets[-1]
        self.id_capacity = id_capacity
        self.waiting = collections.deque()
        self.rejected = []

    def offer(self, req):
        if len(req.sets) > self.max_slots or req.n_ids > self.id_capacity or not req.sets:
            req.error = "request larger than one batch"
            self.rejected.append(req)
            return False
        self.waiting.append(req)
        return True

    def next_batch(self, now):
        """Admit arrived requests in order while they fit; returns
        (requests, bucket) or ([], 0)."""
        reqs = []
        slots = ids = 0
        while self.waiting and self.waiting[0].arrival <= now:
            r = self.waiting[0]
            if slots + len(r.sets) > self.max_slots or ids + r.n_ids > self.id_capacity:
                break
            reqs.append(self.waiting.popleft())
            slots += len(r.sets)
            ids += r.n_ids
        if not reqs:
            return [], 0
        bucket = next(b for b in self.buckets if b >= slots)
        return reqs, bucket

    def pending(self):
        return len(self.waiting)


def id_capacity_from_free_memory(free_bytes, n_lanes, reserve_frac=0.25, max_ids=1 << 24):
    """IDs one lane's device buffer may hold: the free device memory
    `free_bytes` (read after the resident collection and every lane's fixed
    buffers and plan scratch exist) minus a reserve fraction, split evenly
    over `n_lanes`, at 4 bytes per ID, capped at `max_ids` (the pinned host
    staging buffer has the same size).  0 when nothing is left; the batcher
    then rejects every request that carries IDs."""
    if n_lanes < 1 or not 0.0 <= reserve_frac < 1.0:
        raise ValueError("n_lanes >= 1 and 0 <= reserve_frac < 1")
    usable = int(max(0, free_bytes) * (1.0 - reserve_frac)) // n_lanes
    return int(max(0, min(max_ids, usable // 4)))


def pack_batch(reqs, bucket, h_ids, h_off):
    """Write the batch's sets into pinned host buffers (padding sets are
    empty); returns (n_ids, owner) with owner[q] = (request, local index)."""
    pos = 0
    q = 0
    owner = []
    h_off[0] = 0
    for r in reqs:
        for j, s in enumerate(r.sets):
            n = len(s)
            h_ids[pos:pos + n] = s.view(np.int32)
            pos += n
            q += 1
            h_off[q] = pos
            owner.append((r, j))
    h_off[q + 1:bucket + 1] = pos
    return pos, owner


class GpuExecutor:
    """`n_streams` streams, one plan each, one graph per (stream, bucket).

    id_capacity: IDs per batch; None sizes it from the device's free memory
    (``id_capacity_from_free_memory`` over ``mem_reader()``, by default
    torch.cuda.mem_get_info's free bytes) once every lane's fixed buffers
    and plan scratch exist.  The batcher must use ``self.id_capacity``.
    pair_window: accepted pairs copied back inside the captured graph; a
    batch with more copies the rest when it is retired."""

    def __init__(self, plan_kwargs, planes, n_rows, mode, slot_buckets, id_capacity=None,
                 out_capacity=1 << 14, n_streams=2, device=None, mem_reader=None,
                 reserve_frac=0.25, max_ids=1 << 24, pair_window=256):
        import torch
        self.torch = torch
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.planes = planes
        self.n_rows = n_rows
        self.mode = mode
        self.buckets = sorted(slot_buckets)
        self.cap = out_capacity
        self.window = max(1, min(pair_window, out_capacity))
        self.lanes = []
        mb = self.buckets[-1]
        for _ in range(n_streams):
            plan = hoph.Plan(**plan_kwargs)
            lane = dict(plan=plan, stream=torch.cuda.Stream(device=self.dev), busy=None)
            lane["d_off"] = torch.zeros(mb + 1, dtype=torch.int64, device=self.dev)
            lane["out"] = torch.empty((self.cap, 2), dtype=torch.int64, device=self.dev)
            lane["cnt"] = torch.zeros(1, dtype=torch.int64, device=self.dev)
            lane["h_off"] = torch.zeros(mb + 1, dtype=torch.int64).pin_memory()
            lane["h_out"] = torch.empty((self.cap, 2), dtype=torch.int64).pin_memory()
            lane["h_cnt"] = torch.zeros(1, dtype=torch.int64).pin_memory()
            lane["qb"] = {b: torch.empty((plan.G, b, plan.kg), dtype=torch.int32,
                                         device=self.dev) for b in self.buckets}
            lane["graphs"] = {}
            # one eager step of empty sets at the largest batch size sizes the
            # plan's scratch and tables (they depend on the batch size, not the IDs)
            lane["d_ids"] = torch.empty(1, dtype=torch.int32, device=self.dev)
            with torch.cuda.stream(lane["stream"]):
                self._device_step(lane, mb, lane["stream"])
            lane["stream"].synchronize()
            self.lanes.append(lane)
        if id_capacity is None:
            torch.cuda.synchronize(self.dev)
            free = (mem_reader() if mem_reader is not None
                    else torch.cuda.mem_get_info(self.dev)[0])
            id_capacity = id_capacity_from_free_memory(free, n_streams, reserve_frac, max_ids)
        self.id_capacity = int(id_capacity)
        for lane in self.lanes:
            lane["d_ids"] = torch.empty(max(self.id_capacity, 1), dtype=torch.int32,
                                        device=self.dev)
            lane["h_ids"] = torch.empty(max(self.id_capacity, 1), dtype=torch.int32).pin_memory()
        # largest batch first: its eager call sizes the plan's scratch for every
        # bucket, so the scratch never grows (and moves) under a graph that
        # was already captured
        for lane in self.lanes:
            for b in reversed(self.buckets):
                lane["graphs"][b] = self._capture(lane, b)

    def _device_step(self, lane, bucket, stream):
        """Sketch the batch's sets, query them, copy count and pairs back
        (the part of a batch that replays as a graph)."""
        plan = lane["plan"]
        planes_q = lane["qb"][bucket]
        hoph.oph_build_sketches(plan.handle, lane["d_ids"], lane["d_off"], bucket, planes_q,
                                stream)
        hoph.hoph_query_batch(plan.handle, self.mode, planes_q, bucket, self.planes, self.n_rows,
                              lane["out"], self.cap, lane["cnt"], None, stream)
        lane["h_cnt"].copy_(lane["cnt"], non_blocking=True)
        lane["h_out"][:self.window].copy_(lane["out"][:self.window], non_blocking=True)

    def _capture(self, lane, bucket):
        torch = self.torch
        lane["d_off"].zero_()
        s = lane["stream"]
        with torch.cuda.stream(s):
            self._device_step(lane, bucket, s)  # sizes scratch and tables outside capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self._device_step(lane, bucket, s)
        s.synchronize()
        return g

    def free_lane(self):
        for lane in self.lanes:
            if lane["busy"] is None:
                return lane
        return None

    def launch(self, lane, reqs, bucket):
        n_ids, owner = pack_batch(reqs, bucket, lane["h_ids"].numpy(), lane["h_off"].numpy())
        s = lane["stream"]
        with self.torch.cuda.stream(s):
            # exactly this batch's bytes go over, then the captured device work
            if n_ids:
                lane["d_ids"][:n_ids].copy_(lane["h_ids"][:n_ids], non_blocking=True)
            lane["d_off"][:bucket + 1].copy_(lane["h_off"][:bucket + 1], non_blocking=True)
            lane["graphs"][bucket].replay()
            ev = self.torch.cuda.Event()
            ev.record(s)
        lane["busy"] = (reqs, owner, ev)

    def poll(self, now_fn, block=False):
        """Retire finished batches; returns the requests completed."""
        done = []
        for lane in self.lanes:
            if lane["busy"] is None:
                continue
            reqs, owner, ev = lane["busy"]
            if block:
                ev.synchronize()
            elif not ev.query():
                continue
            rc = hoph.hoph_sync_status(lane["plan"].handle, lane["stream"])
            n = int(lane["h_cnt"][0])
            if min(n, self.cap) > self.window:  # the pairs past the captured window
                m = min(n, self.cap)
                lane["h_out"][self.window:m].copy_(lane["out"][self.window:m])
            t = now_fn()
            err = None
            if rc not in (hoph.HOPH_OK,):
                err = hoph.hoph_status_string(rc)
            pairs = lane["h_out"].numpy()[:min(n, self.cap)].view(hoph.PAIR_DTYPE).reshape(-1)
            per = {id(r): [] for r in reqs}
            for p in pairs:
                qi = int(p["query"])
                if qi < len(owner):
                    r, j = owner[qi]
                    per[id(r)].append((j, int(p["row"]), int(p["groups"]), int(p["matches"])))
            for r in reqs:
                r.pairs = sorted(per[id(r)])
                r.done = t
                r.error = err
                done.append(r)
            lane["busy"] = None
        return done

    def close(self):
        for lane in self.lanes:
            lane["plan"].close()


def serve(executor, batcher, requests, clock=time.perf_counter, spin=True):
    """Play `requests` (sorted by arrival, relative seconds) through the
    service in real time; returns the completed requests."""
    t0 = clock()
    now = lambda: clock() - t0  # noqa: E731
    pending = collections.deque(requests)
    completed = []
    while pending or batcher.pending() or any(l["busy"] for l in executor.lanes):
        t = now()
        while pending and pending[0].arrival <= t:
            batcher.offer(pending.popleft())
        completed += executor.poll(now)
        lane = executor.free_lane()
        if lane is not None:
            reqs, bucket = batcher.next_batch(t)
            if reqs:
                executor.launch(lane, reqs, bucket)
                continue
        if not spin:
            time.sleep(20e-6)
    completed += batcher.rejected
    return completed


def latency_summary(completed):
    lat = np.asarray([r.done - r.arrival for r in completed if r.done is not None])
    if not len(lat):
        return {}
    return {"requests": int(len(lat)), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}


def poisson_requests(rate_qps, duration_s, seed, size_fn, max_sets=256):
    """Requests of U[1, max_sets] query sets, Poisson arrivals at rate_qps
    query sets per second (request rate = rate_qps / mean sets per request)."""
    rng = np.random.default_rng(seed)
    mean_sets = (1 + max_sets) / 2
    lam = rate_qps / mean_sets
    t = 0.0
    reqs = []
    rid = 0
    while True:
        t += rng.exponential(1.0 / lam)
        if t > duration_s:
            break
        n = int(rng.integers(1, max_sets + 1))
        reqs.append(Request(rid, size_fn(rng, n), t))
        rid += 1
    return reqs
