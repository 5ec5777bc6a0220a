"""Autotuner of hoph_query_batch execution knobs.

Knobs (hoph_exec: strategy, consumer warps, pipeline stages, tile rows,
CTAs per SM) change how the comparison is scheduled, never its result: the
method's k' and layout are fixed by the plan.  The tuner times each
candidate setting with CUDA events on the caller's stream, checks that
every setting returns the same accepted pairs, and leaves the fastest one
set on the plan.  Results are cached per (plan, mode, batch shape).
"""
import numpy as np

from . import hoph

_cache = {}

QUERY_DEFAULTS = dict(strategy=-1, tile_rows=0, consumer_warps=0, ctas_per_sm=0, stages=0,
                      lanes_per_row=0)
JOIN_CANDIDATES = [dict(strategy=1, lanes_per_row=l, consumer_warps=c, stages=s)
                   for l, c, s in ((0, 16, 2), (0, 12, 2), (0, 8, 3), (0, 16, 3), (-2, 16, 2),
                                   (-2, 16, 3), (-2, 16, 4), (-2, 31, 2), (-2, 24, 2))]
# the striped-map filter (lanes over a row's bins): warps x stages x rows per tile
# (0: a 64 KB stage)
JOIN_CANDIDATES += [dict(strategy=1, lanes_per_row=32, consumer_warps=c, stages=s, tile_rows=r)
                    for c, s, r in ((16, 2, 0), (16, 3, 0), (16, 3, 256), (16, 4, 256),
                                    (8, 3, 256), (12, 3, 384))]
DENSE_CANDIDATES = [dict(strategy=0, consumer_warps=c, stages=s, tile_rows=r)
                    for c, s, r in ((8, 4, 0), (15, 4, 0), (8, 6, 0), (4, 4, 0), (15, 2, 64),
                                    (8, 4, 32), (15, 3, 32), (8, 2, 64), (4, 8, 16), (6, 4, 32))]


def _lanes(cand, W):
    """lanes_per_row 0 = one lane per 32 bins, -2 = one lane per 16 bins."""
    cand = dict(cand)
    if cand.get("lanes_per_row", 0) == -2:
        cand["lanes_per_row"] = max(1, W // 16)
    return cand


def tune_query(plan, mode, q_planes, n_queries, c_planes, n_rows, out, capacity, count,
               stream=None, reps=3, candidates=None, finalists=3, rounds=4):
    """Pick the fastest execution setting for this batch shape; returns
    (best setting, {setting index: ms}).  Every candidate is timed once; the
    `finalists` fastest are then timed again, interleaved, `rounds` times,
    and the lowest median wins (one short timing per candidate cannot tell
    settings a few percent apart).  Compact (16-bit) planes go through
    hoph_query_batch16."""
    import torch
    call = hoph.hoph_query_batch16 if c_planes.element_size() == 2 else hoph.hoph_query_batch
    key = (plan.handle, mode, n_queries, n_rows, plan.k, plan.kg, c_planes.element_size())
    if key in _cache:
        best = _cache[key]
        plan.update_exec(**{**QUERY_DEFAULTS, **best})
        return best, {}
    if candidates is None:
        candidates = JOIN_CANDIDATES + DENSE_CANDIDATES if n_queries >= 16 else DENSE_CANDIDATES
    stream = stream or torch.cuda.current_stream()
    times = {}
    ref = None
    best = None
    tried = {}
    W = plan.k if mode in (0, "oph_full") else plan.kg

    def timed(cand):
        plan.update_exec(**{**QUERY_DEFAULTS, **cand})
        call(plan.handle, mode, q_planes, n_queries, c_planes, n_rows, out, capacity, count,
             None, stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            call(plan.handle, mode, q_planes, n_queries, c_planes, n_rows, out, capacity, count,
                 None, stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    for i, cand in enumerate(candidates):
        cand = _lanes(cand, W)
        if cand["strategy"] == 0 and n_queries >= 256 and n_rows >= 1 << 20:
            continue  # dense at large batches is tens of times slower; skip
        try:
            plan.update_exec(**{**QUERY_DEFAULTS, **cand})
            call(plan.handle, mode, q_planes, n_queries, c_planes, n_rows, out, capacity, count,
                 None, stream)
        except hoph.HophError:
            continue  # setting not available for this shape
        stream.synchronize()
        n = int(count.item())
        got = out[:min(n, capacity)].cpu().numpy().copy()
        if ref is None:
            ref = (n, got)
        elif n != ref[0] or not np.array_equal(got, ref[1]):
            raise RuntimeError("execution setting %r changed the result" % cand)
        times[i] = timed(cand)
        tried[i] = cand
    if len(tried) > 1 and finalists > 1 and rounds > 0:
        top = sorted(tried, key=times.get)[:finalists]
        runs = {i: [] for i in top}
        for _ in range(rounds):
            for i in top:
                runs[i].append(timed(tried[i]))
        for i in top:
            times[i] = float(np.median(runs[i]))
        best_i = min(top, key=times.get)
        best = tried[best_i]
    elif tried:
        best = tried[min(tried, key=times.get)]
    if best is None:
        plan.update_exec(**QUERY_DEFAULTS)
        return None, times
    plan.update_exec(**{**QUERY_DEFAULTS, **best})
    _cache[key] = best
    return best, times


SKETCH_CANDIDATES = (0, 10, 11, 12, 13, 14, 64)


def tune_sketch(plan, d_ids, d_offsets, n_sets, out, stream=None, reps=3,
                candidates=SKETCH_CANDIDATES, finalists=3, rounds=4):
    """Pick the size (bits of a set's ID count) from which a set gets a whole
    CTA instead of one warp, for this batch; 0 is the library's own choice,
    64 warps only.  Every setting must give the same sketches.  Returns
    (best bits, {bits: ms})."""
    import torch
    key = ("sketch", plan.handle, n_sets, out.element_size())
    if key in _cache:
        plan.update_exec(sketch_cta_bits=_cache[key])
        return _cache[key], {}
    stream = stream or torch.cuda.current_stream()
    call = hoph.oph_build_sketches16 if out.element_size() == 2 else hoph.oph_build_sketches

    def timed(bits):
        plan.update_exec(sketch_cta_bits=bits)
        call(plan.handle, d_ids, d_offsets, n_sets, out, stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            call(plan.handle, d_ids, d_offsets, n_sets, out, stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    times, ref = {}, None
    for bits in candidates:
        plan.update_exec(sketch_cta_bits=bits)
        call(plan.handle, d_ids, d_offsets, n_sets, out, stream)
        stream.synchronize()
        got = out.cpu()
        if ref is None:
            ref = got
        elif not torch.equal(got, ref):
            raise RuntimeError("sketch_cta_bits=%d changed the sketches" % bits)
        times[bits] = timed(bits)
    # the closest settings again, interleaved (as for the query knobs)
    top = sorted(times, key=times.get)[:finalists]
    runs = {b: [] for b in top}
    for _ in range(rounds if len(top) > 1 else 0):
        for b in top:
            runs[b].append(timed(b))
    for b in top:
        if runs[b]:
            times[b] = float(np.median(runs[b]))
    best = min(top, key=times.get)
    plan.update_exec(sketch_cta_bits=best)
    _cache[key] = best
    return best, times
