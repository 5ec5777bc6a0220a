#!/usr/bin/env python
"""Benchmark of the batched (a:b)HOPH query path on GB300.

Workload (one step): sketch a batch of 1,024 query sets (K1, OPH/HOPH
sketching) and compare them with (1:2)HOPH, k = 256, k' = 64, T = 0.7,
eps = 1e-4 against a device-resident collection of 10,000,000 sketches
(10.24 GB; sets of lognormal size, median 300, sigma 1, clipped to
[10, 20000], uniform IDs over D = 2^20).  10% of the queries are planted
near duplicates (Jaccard 0.6-0.95) of collection rows, the rest are fresh
random sets.  value = (query, row) sketch-pair comparisons per second.

Also reported on the same line: batched sketching of 1,000,000 sets
(lognormal sizes, Zipf(1.1) IDs, k = 256 OPH) as sets/s and GB/s, the
roofline fraction of the dominant kernel from live CUDA events, the CPU
oracle timed on this host, an end-to-end number through host buffers,
recall/precision of the planted near duplicates against exact Jaccard and
the one-query-per-launch full-scan OPH baseline.

--impl reference times the CPU oracle itself on a bounded sample per step.
"""
import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HOPH sketch-pair comparisons/sec + sets sketched/sec, % HBM roofline, equal recall"
UNIT = "pair-comparisons/s"
D = 1 << 20
K, KG, AB = 256, 64, (1, 2)
T, EPS = (7, 10), 1e-4
PERM_SEED, COLL_SEED, Q_SEED, PLANT_SEED = 1, 11, 12, 13
SKETCH_SEED = 21
# output capacity (accepted pairs) of a 1,024-query step: about 70 pairs are
# accepted per batch; up to 65,536 the library sorts them in one CTA
CAP = 1 << 16

# dram read+write bytes per filter-kernel launch from an ncu capture, keyed by
# the sha256 of the filter kernel's source it was taken on (null once that
# source changes)
NCU_TRAFFIC = {"e0b00ae8eed0effc": 2575.74e6}  # 2*10^6-row capture x 5 rows
# the same for the striped filter over compact 16-bit planes (its own source)
NCU_TRAFFIC_STRIPED = {"8fa6ac907bca01c7": 1297.26e6}  # 2*10^6-row capture x 5 rows
# DRAM bytes of the 10^6-set sketch call (both launches), keyed to sketch.cu's hash
NCU_TRAFFIC_SKETCH = {"000757fea3813741": 3184.5e6}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--rows", type=int, default=10_000_000)
    p.add_argument("--queries", type=int, default=1024)
    p.add_argument("--sketch-sets", type=int, default=1_000_000)
    p.add_argument("--e2e-steps", type=int, default=100)
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-extras", action="store_true", help="skip sketch/OPH/CPU legs")
    p.add_argument("--in-flight", type=int, default=8,
                   help="batches in flight in the timed schedule (each lane its own plan, "
                        "stream branch and query batch)")
    p.add_argument("--decision-thr", default="697/1000",
                   help="decision threshold of the timed HOPH step; ground truth stays "
                        "Jaccard >= 7/10.  697/1000 is where (1:2)HOPH's recall on this "
                        "seeded workload reaches plain OPH's at 7/10 (re-checked every run "
                        "by the recall study)")
    p.add_argument("--no-truth-threshold", action="store_true",
                   help="skip timing the same schedule at the ground-truth threshold 7/10")
    p.add_argument("--details", default=None,
                   help="also write the studies' JSON to this file")
    p.add_argument("--profile", nargs="?", const="query",
                   choices=("query", "sketch", "oph1", "self_join", "shingle"),
                   help="few launches of the query step (or of the 10^6-set sketch, of the "
                        "one-query OPH full scan with its tuned knobs, or one self-join of "
                        "the first --rows rows), for ncu")
    p.add_argument("--profile-knobs", default="",
                   help="execution knobs of the profiled query step, e.g. "
                        "'strategy=1,lanes_per_row=32,stages=2,tile_rows=256'")
    p.add_argument("--profile-compact", action="store_true",
                   help="profile the query step over compact (uint16) planes")
    p.add_argument("--no-graph", action="store_true", help="eager launches instead of a graph")
    p.add_argument("--no-pipeline", action="store_true",
                   help="one batch at a time (no second batch in flight on a second stream)")
    p.add_argument("--no-tune", action="store_true", help="library default execution knobs")
    p.add_argument("--no-serve", action="store_true", help="skip the serving sweep")
    p.add_argument("--no-compact", action="store_true",
                   help="skip the same step over compact (uint16) sketch planes")
    p.add_argument("--no-self-join", action="store_true",
                   help="skip the all-pairs self-join of a 10^6-row collection")
    p.add_argument("--no-sweep", action="store_true",
                   help="skip the threshold / tolerance sweep on the 5,000-set workload")
    p.add_argument("--serve-rates", default="2000,20000,100000,150000",
                   help="Poisson arrival rates (query sets per second)")
    p.add_argument("--serve-seconds", type=float, default=1.5)
    p.add_argument("--no-shingle", action="store_true", help="skip the D=2^32 shingle workload")
    p.add_argument("--shingle-rows", type=int, default=5_000_000)
    p.add_argument("--shingle-queries", type=int, default=100_000)
    return p.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def sketch_src_sha():
    """sha256[:16] of the sketch kernels' source file."""
    with open(os.path.join(ROOT, "paper_1805_11254_gb300", "csrc", "sketch.cu")) as f:
        return hashlib.sha256(f.read().encode()).hexdigest()[:16]


def filter_src_sha(striped=False):
    """sha256[:16] of the join filter's source: FilterArgs through
    filter_kernel, and for the striped filter on to its end."""
    with open(os.path.join(ROOT, "paper_1805_11254_gb300", "csrc", "query.cu")) as f:
        text = f.read()
    a = text.index("struct FilterArgs {")
    b = text.index("// Join filter over a striped group map")
    if striped:
        b = text.index("// Join strategy, part 3")
    return hashlib.sha256(text[a:b].encode()).hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

def collection_host(n_rows, rank):
    from paper_1805_11254_gb300 import synth
    sizes = synth.counter_collection_sizes(n_rows, COLL_SEED + 1000 * rank)
    return synth.offsets_from_sizes(sizes), COLL_SEED + rank


def query_sets(n_q, off, coll_seed):
    from paper_1805_11254_gb300 import synth
    return synth.query_batch(n_q, 0.1, D, coll_seed, off, 0.6, 0.95, Q_SEED, PLANT_SEED)


def to_dev(a, dev):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).to(dev)


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------

def cpu_oracle_pass(qw, off, coll_seed, rows, threads, lo, perm, z, thr=T):
    """One bounded CPU step: oracle sketches of the query batch and the
    (1:2)HOPH comparison against `rows` collection rows.  The sample rows'
    sketches are prepared outside the timing (the collection is resident on
    both sides).  Returns (seconds, pairs)."""
    from oracle import oracle_c as oc
    from paper_1805_11254_gb300 import synth
    ids = synth.counter_ids(coll_seed, 0, int(off[rows]), D)
    c_sk = oc.sketch(ids, off[:rows + 1], lo, perm=perm, threads=threads)
    t0 = time.perf_counter()
    q_sk = oc.sketch(qw["q_ids"], qw["q_off"], lo, perm=perm, threads=threads)
    oc.query("hoph", q_sk, c_sk, KG, thr[0], thr[1], EPS, z=z, threads=threads)
    return time.perf_counter() - t0, len(qw["q_off"]) - 1


def cpu_baseline(qw, off, coll_seed, target_s, n_rows, thr=T):
    from oracle import oracle_c as oc
    threads = os.cpu_count() or 1
    lo = oc.layout(D, K, KG, *AB)
    perm = oc.permutation(D, PERM_SEED)
    z = np.diff(lo[::KG]).astype(np.uint64)
    probe = min(2000, n_rows)
    t, nq = cpu_oracle_pass(qw, off, coll_seed, probe, threads, lo, perm, z, thr)
    rows = int(min(n_rows, max(probe, probe * target_s / max(t, 1e-6))))
    t, nq = cpu_oracle_pass(qw, off, coll_seed, rows, threads, lo, perm, z, thr)
    # one core, small sample
    t1, _ = cpu_oracle_pass(qw, off, coll_seed, probe, 1, lo, perm, z, thr)
    return {"value": nq * rows / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "cpu_model": cpu_model(), "value_one_core": nq * probe / t1,
            "sample": "C oracle: sketch %d query sets + (1:2)HOPH vs rows 0..%d (%d pairs, "
                      "%.1f s); one core: rows 0..%d" % (nq, rows - 1, nq * rows, t, probe - 1)}


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo or lscpu), for the record."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    from oracle import oracle_c as oc
    oc.build()
    off, coll_seed = collection_host(args.rows, 0)
    qw = lane_batch(args, off, coll_seed, 0)
    thr = decision_thr(args)
    threads = os.cpu_count() or 1
    lo = oc.layout(D, K, KG, *AB)
    perm = oc.permutation(D, PERM_SEED)
    z = np.diff(lo[::KG]).astype(np.uint64)
    budget = 150.0 / max(1, args.steps + args.warmup)  # seconds per step
    probe = 256
    t, nq = cpu_oracle_pass(qw, off, coll_seed, probe, threads, lo, perm, z, thr)
    rows = int(min(args.rows, max(16, probe * budget / max(t, 1e-6))))
    for _ in range(args.warmup):
        cpu_oracle_pass(qw, off, coll_seed, rows, threads, lo, perm, z, thr)
    total = 0.0
    for _ in range(args.steps):
        t, nq = cpu_oracle_pass(qw, off, coll_seed, rows, threads, lo, perm, z, thr)
        total += t
    value = nq * rows * args.steps / total
    sample = ("per step: C oracle sketches %d query sets + (1:2)HOPH vs collection rows "
              "0..%d (%d pairs)" % (nq, rows - 1, nq * rows))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(headline_json(line), flush=True)


def decision_thr(args):
    """The decision threshold of the timed step as (num, den)."""
    num, den = (int(x) for x in args.decision_thr.split("/"))
    return num, den


def workload_config(args, world):
    thr = decision_thr(args)
    return {"workload": "step = sketch %d query sets (10%% planted near duplicates) + "
                        "(1:2)HOPH query vs %d resident k=256 sketches/GPU"
                        % (args.queries, args.rows),
            "D": D, "k": K, "k_group": KG, "a_b": "1:2", "T_truth": "%d/%d" % T,
            "T_decision": "%d/%d" % thr, "eps": EPS, "queries": args.queries,
            "rows_per_gpu": args.rows, "sets": "lognormal(300,1) [10,20000], uniform IDs",
            "l2": "inputs > L2 (2.56 GB plane/pass)",
            "schedule": "%d batches in flight" % max(1, args.in_flight),
            "parallelism": "rows sharded x%d, no data-path collective" % world}


# ---------------------------------------------------------------------------
# native
# ---------------------------------------------------------------------------

def lane_batch(args, off, coll_seed, lane):
    """The query batch of in-flight lane `lane` (lane 0: the step's batch;
    every other lane draws its own sets with its own seeds)."""
    from paper_1805_11254_gb300 import synth
    return synth.query_batch(args.queries, 0.1, D, coll_seed, off, 0.6, 0.95,
                             Q_SEED + 1000 * lane, PLANT_SEED + 1000 * lane)


def run_native(args):
    import torch
    from paper_1805_11254_gb300 import build_lib, hoph, shard
    rank, world, local = env_rank()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    if rank == 0:  # one rank compiles (when the library is not up to date), all load it
        build_lib.build()
    barrier()
    hoph.load()
    stream = torch.cuda.current_stream()
    thr = decision_thr(args)

    def max_over_ranks(x):
        return shard.max_over_ranks(x, device=dev)

    if args.profile == "sketch":
        sketch_leg(dev, stream, measured_peaks()[0], steps=2)
        return
    if args.profile == "shingle":
        profile_shingle(args, dev, stream)
        return

    # ---- collection (setup, untimed)
    off, coll_seed = collection_host(args.rows, rank)
    if args.profile == "oph1":
        profile_oph1(args, off, coll_seed, dev, stream)
        return
    if args.profile == "self_join":
        profile_self_join(args, off, coll_seed, dev, stream)
        return
    n_ids = int(off[-1])
    with hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=thr, epsilon=EPS) as plan:
        d_off = to_dev(off, dev)
        d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(coll_seed, 0, n_ids, D, 0, None, 0, d_ids)
        planes = plan.sketch(d_ids, d_off, args.rows)
        plan.check()
        coll_sketch = None
        if rank == 0 and world == 1 and not args.no_extras and not args.profile:
            # the same call again, timed: 10^7 sets of uniform IDs over 2^20 (next to
            # no repeated IDs within a set, unlike the Zipf sketch workload)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                plan.sketch(d_ids, d_off, args.rows, out=planes)
            e1.record(stream)
            torch.cuda.synchronize()
            plan.check()
            ms = e0.elapsed_time(e1) / 2
            b = 4 * n_ids + 8 * (args.rows + 1) + 4 * K * args.rows
            # every ID is one random 4-byte gather from the 4 MiB psi table, and the
            # L1 serves one cache line per SM clock: a floor for the call
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            gather_ms = n_ids / (sms * 2070e6) * 1e3
            coll_sketch = {"sets": args.rows, "ids": n_ids, "ms_per_call": ms,
                           "sets_per_s": args.rows / (ms / 1e3),
                           "hbm_frac": b / (ms / 1e3) / 1e9 / measured_peaks()[0]["hbm_gbs"],
                           "gather_floor_ms": gather_ms, "gather_floor_frac": gather_ms / ms,
                           "how": "the collection's own sketch call (uniform IDs over 2^20), "
                                  "timed twice after the setup call; gather floor = one L1 "
                                  "line per ID at one line per SM per clock (2,070 MHz)"}
    del d_ids, d_off
    torch.cuda.empty_cache()

    n_lanes = max(1, args.in_flight)
    batches = [lane_batch(args, off, coll_seed, ln) for ln in range(n_lanes)]
    qw = batches[0]

    if args.profile:
        with hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=thr, epsilon=EPS) as p:
            if args.profile_knobs:
                p.set_exec(**{kv.split("=")[0]: int(kv.split("=")[1])
                              for kv in args.profile_knobs.split(",")})
            dq_ids, dq_off = to_dev(qw["q_ids"], dev), to_dev(qw["q_off"], dev)
            build, query, dt = hoph.oph_build_sketches, hoph.hoph_query_batch, torch.int32
            c = planes
            if args.profile_compact:
                build, query, dt = hoph.oph_build_sketches16, hoph.hoph_query_batch16, torch.int16
                d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
                hoph.hoph_synth_ids(coll_seed, 0, n_ids, D, 0, None, 0, d_ids)
                c = p.sketch16(d_ids, to_dev(off, dev), args.rows)
                del d_ids, planes
            q = torch.empty((p.G, args.queries, KG), dtype=dt, device=dev)
            out = torch.empty((CAP, 2), dtype=torch.int64, device=dev)
            cnt = torch.zeros(1, dtype=torch.int64, device=dev)
            for _ in range(max(1, args.warmup)):
                build(p.handle, dq_ids, dq_off, args.queries, q, stream)
                query(p.handle, hoph.HOPH_MODE_HOPH, q, args.queries, c, args.rows, out, CAP, cnt,
                      None, stream)
            p.check()
            print(json.dumps({"profiled": "query", "knobs": p.exec_kwargs,
                              "compact": bool(args.profile_compact),
                              "accepted": int(cnt.item())}), flush=True)
        return

    peaks, peak_kind = measured_peaks()
    head = headline_leg(args, planes, batches, dev, stream, thr, barrier, max_over_ranks, local,
                        truth_threshold_too=not (args.no_extras or args.no_truth_threshold))
    value = head["value"]
    line = headline_line(args, world, head, peaks, peak_kind)
    details = {"headline": {k_: v for k_, v in head.items() if k_ not in ("pairs", "roofline")}}

    if not args.no_extras:  # every rank: the end-to-end step is timed over all of them
        def sync(x):
            barrier()
            return max_over_ranks(x)
        e2e = e2e_leg(args, thr, batches, planes, dev, world, sync)
        line["e2e"] = {k_: e2e[k_] for k_ in ("value", "unit", "h2d_bytes_per_step",
                                              "d2h_bytes_per_step", "ms_per_step")}
        details["e2e"] = e2e
    # the other legs are single-GPU studies: rank 0 of a one-GPU run only
    if rank == 0 and world == 1 and not args.no_extras:
        details["sketch"] = sketch_leg(dev, stream, peaks)
        details["sketch"]["uniform_ids_collection"] = coll_sketch
        rq = recall_queries(off, coll_seed)
        details["oph_full_scan_baseline"], oph_pairs, oph_rq_pairs = oph_baseline_leg(
            args, off, coll_seed, qw, dev, stream, value, rq)
        details["quality"] = quality(qw, {"hoph": head["pairs"], "oph_full_scan": oph_pairs},
                                     off, coll_seed, args)
        dq_ids, dq_off = to_dev(qw["q_ids"], dev), to_dev(qw["q_off"], dev)
        nq = args.queries
        eps_runs = eps_variants(args, planes, dq_ids, dq_off, nq, dev, stream, rq)
        thr_set = sorted(set(EQUAL_RECALL_T) | {thr}, key=lambda t: -t[0] / t[1])
        thr_runs = eps_variants(args, planes, dq_ids, dq_off, nq, dev, stream, rq,
                                variants=[(t, EPS) for t in thr_set])
        methods = {"oph_full_scan": oph_rq_pairs}
        methods.update({"hoph_eps_%g" % e: r["pairs"] for e, r in eps_runs.items()})
        methods.update({"hoph_T_%d_%d" % t: r["pairs"] for t, r in thr_runs.items()})
        study = quality(rq, methods, off, coll_seed, args, n_random_rows=500)
        er = equal_recall(study, eps_runs, nq, args.rows, len(rq["q_off"]) - 1, thr_runs)
        m_thr = study["hoph_T_%d_%d" % thr]
        er["headline_decision_threshold"] = "%d/%d" % thr
        er["headline_recall"] = m_thr["recall"]
        er["headline_precision"] = m_thr["precision"]
        er["headline_at_equal_recall"] = m_thr["recall"] >= er["oph_full_scan_recall"]
        details["equal_recall"] = er
        line["cpu_baseline"] = cpu_baseline(qw, off, coll_seed, args.cpu_seconds, args.rows, thr)
        if not args.no_serve:
            details["serving"] = serving_leg(args, planes, dev, details["oph_full_scan_baseline"])
        if not args.no_compact:
            details["compact"] = compact_leg(args, off, coll_seed, dq_ids, dq_off, nq,
                                             head["pairs"], dev, stream, peaks, thr)
        if not args.no_sweep:
            details["sweeps"] = sweep_leg(dev, stream)
            details["large_output"] = large_output_leg(dev, stream)
        if not args.no_self_join:
            details["self_join"] = self_join_leg(off, coll_seed, dev, stream)
        if not args.no_shingle:
            del planes
            torch.cuda.empty_cache()
            details["shingle"] = shingle_leg(args, dev, stream, peaks)
        line["metric_parts"] = metric_parts(details)
    if rank == 0:
        emit(line, details, args.details)
    if world > 1:
        torch.distributed.destroy_process_group()


def headline_line(args, world, head, peaks, peak_kind):
    """The benchmark's JSON line from the timed step's results (the e2e,
    cpu_baseline and metric_parts keys are added by the caller)."""
    roofline = dict(head["roofline"])
    roofline["peak"] = peaks["hbm_gbs"]
    roofline["frac"] = roofline["achieved"] / peaks["hbm_gbs"]
    roofline["peak_source"] = "%s hbm_gbs (copy)" % peak_kind
    return {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": workload_config(args, world),
            "roofline": roofline, "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"]}


def metric_parts(details):
    """The metric's other parts, in a few numbers: sets sketched per second,
    the sketch's HBM fraction, the recalls behind "equal recall", and the
    plain-OPH baseline the HOPH step is compared with."""
    parts = {}
    sk = details.get("sketch")
    if sk:
        parts["sets_sketched_per_s"] = sk["sets_per_s"]
        parts["sketch_hbm_frac"] = sk["roofline"]["frac"]
    er = details.get("equal_recall")
    if er:
        parts["recall_hoph"] = er["headline_recall"]
        parts["recall_oph_full_scan"] = er["oph_full_scan_recall"]
        parts["at_equal_recall"] = er["headline_at_equal_recall"]
    ob = details.get("oph_full_scan_baseline")
    if ob:
        parts["oph_one_query_per_launch_pairs_per_s"] = ob["value"]
    h = details.get("headline", {})
    if "value_at_T" in h:
        parts["value_at_T_7_10"] = h["value_at_T"]
    return parts


def emit(line, details, details_path=None):
    """Print the headline as the one JSON line on stdout (kept short); the
    studies go to stderr as one line prefixed 'details: ' and, when asked,
    to a file."""
    text = json.dumps(details, default=_jsonable)
    if details_path:
        d = os.path.dirname(os.path.abspath(details_path))
        os.makedirs(d, exist_ok=True)
        with open(details_path, "w") as f:
            f.write(text + "\n")
    print("details: " + text, file=sys.stderr, flush=True)
    print(headline_json(line), flush=True)


def _jsonable(x):
    if isinstance(x, (np.integer,)):
        return int(x)
    if isinstance(x, (np.floating,)):
        return float(x)
    if isinstance(x, np.ndarray):
        return x.tolist()
    return str(x)


def _round(x):
    """Floats to 6 significant digits (the line stays short)."""
    if isinstance(x, float):
        return float("%.6g" % x)
    if isinstance(x, dict):
        return {k_: _round(v) for k_, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_round(v) for v in x]
    return x


HEADLINE_MAX_BYTES = 2048
# what goes first if a line would still be too long (never the contract's keys)
_TRIM = (("metric_parts",), ("cpu_baseline", "cpu_model"), ("config", "sets"), ("config", "l2"),
         ("roofline", "peak_source"), ("cpu_baseline", "sample"), ("config", "workload"))


def headline_json(line):
    """The headline as one JSON line under 2 KB: floats rounded to six
    significant digits, no spaces; optional keys are dropped (in _TRIM's
    order) if it would still be longer."""
    line = _round(line)
    text = json.dumps(line, default=_jsonable, separators=(",", ":"))
    for path in _TRIM:
        if len(text) <= HEADLINE_MAX_BYTES:
            break
        d = line
        for key in path[:-1]:
            d = d.get(key, {}) if isinstance(d, dict) else {}
        if isinstance(d, dict) and path[-1] in d:
            del d[path[-1]]
            text = json.dumps(line, default=_jsonable, separators=(",", ":"))
    return text


def headline_leg(args, planes, batches, dev, stream, thr, barrier, max_over_ranks, local,
                 knobs=None, truth_threshold_too=True):
    """The timed step: sketch a batch of query sets and (1:2)HOPH-query it
    against the resident collection.  Every in-flight lane has its own plan,
    stream branch and query batch; the step is replayed as a CUDA graph, one
    batch at a time and with all lanes in flight (the headline schedule,
    fixed by --in-flight).  Returns value, timings, roofline inputs and lane
    0's pairs.  `knobs`: execution knobs to use instead of tuning."""
    import torch
    from paper_1805_11254_gb300 import autotune, hoph
    nq = args.queries
    cap = CAP
    lanes = []
    for b in batches:
        p = hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=thr, epsilon=EPS)
        lanes.append(dict(plan=p, ids=to_dev(b["q_ids"], dev), off=to_dev(b["q_off"], dev),
                          q=torch.empty((p.G, nq, KG), dtype=torch.int32, device=dev),
                          out=torch.empty((cap, 2), dtype=torch.int64, device=dev),
                          cnt=torch.zeros(1, dtype=torch.int64, device=dev)))

    def lane_step(ln, s):
        hoph.oph_build_sketches(ln["plan"].handle, ln["ids"], ln["off"], nq, ln["q"], s)
        hoph.hoph_query_batch(ln["plan"].handle, hoph.HOPH_MODE_HOPH, ln["q"], nq, planes,
                              args.rows, ln["out"], cap, ln["cnt"], None, s)

    def lane_pairs(ln):
        c_ = int(ln["cnt"].item())
        return c_, ln["out"][:min(c_, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1).copy()

    l0 = lanes[0]
    best, tune_ms = knobs, {}
    if knobs is not None:
        l0["plan"].set_exec(**knobs)
    elif not args.no_tune:  # tuned on lane 0's own sketches
        hoph.oph_build_sketches(l0["plan"].handle, l0["ids"], l0["off"], nq, l0["q"], stream)
        best, tune_ms = autotune.tune_query(l0["plan"], hoph.HOPH_MODE_HOPH, l0["q"], nq, planes,
                                            args.rows, l0["out"], cap, l0["cnt"], stream)
    for ln in lanes:
        ln["plan"].set_exec(**l0["plan"].exec_kwargs)
        for _ in range(max(3, args.warmup)):  # also sizes scratch outside any capture
            lane_step(ln, stream)
        ln["plan"].check()
        ln["n"], ln["pairs"] = lane_pairs(ln)
    st = torch.zeros(hoph.STATS_WORDS, dtype=torch.int64, device=dev)
    hoph.hoph_query_batch(l0["plan"].handle, hoph.HOPH_MODE_HOPH, l0["q"], nq, planes, args.rows,
                          l0["out"], cap, l0["cnt"], st, stream)
    stats = hoph.hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes())

    # kernels one step launches (the library's own count, one eager step)
    hoph.hoph_plan_enable_timing(l0["plan"].handle, True)
    lane_step(l0, stream)
    _, _, launches_per_step = hoph.hoph_plan_read_timing(l0["plan"].handle)

    # every lane's step is one CUDA graph (timing events inside), captured on
    # the lane's own stream
    for ln in lanes:
        hoph.hoph_plan_enable_timing(ln["plan"].handle, True)
        ln["s"] = torch.cuda.Stream(device=dev)
        ln["s"].wait_stream(stream)
        with torch.cuda.stream(ln["s"]):
            lane_step(ln, ln["s"])
        ln["g"] = torch.cuda.CUDAGraph()
        with torch.cuda.graph(ln["g"], stream=ln["s"]):
            lane_step(ln, ln["s"])
        stream.wait_stream(ln["s"])
    torch.cuda.synchronize()
    for ln in lanes:
        with torch.cuda.stream(ln["s"]):
            ln["g"].replay()
        ln["s"].synchronize()
        ln["plan"].check()
        if lane_pairs(ln)[0] != ln["n"] or not np.array_equal(lane_pairs(ln)[1], ln["pairs"]):
            raise RuntimeError("a graph replay changed a batch's result")

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def run_steps(k, lns):
        """k steps dealt round-robin over the lanes: step i replays lane
        i mod n's graph on that lane's stream, after its previous step only
        (no barrier between steps)."""
        for ln in lns:
            ln["s"].wait_event(e0)
        for i in range(k):
            ln = lns[i % len(lns)]
            with torch.cuda.stream(ln["s"]):
                ln["g"].replay()
        for ln in lns:
            stream.wait_stream(ln["s"])

    def timed(lns):
        clocks = Clocks(local)
        clocks.start()
        time.sleep(0.3)
        # the GPU is kept busy right up to the timed region (untimed steps),
        # so it does not start the region from an idle power state
        ew = torch.cuda.Event()
        ew.record(stream)
        for ln in lns:
            ln["s"].wait_event(ew)
        for i in range(max(2 * len(lns), args.warmup)):
            with torch.cuda.stream(lns[i % len(lns)]["s"]):
                lns[i % len(lns)]["g"].replay()
        for ln in lns:
            stream.wait_stream(ln["s"])
        barrier()
        e0.record(stream)
        run_steps(args.steps, lns)
        e1.record(stream)
        barrier()
        t = max_over_ranks(e0.elapsed_time(e1))
        return t, clocks.stop()

    def phases(lns, rounds):
        """Mean per-launch phase times (ms) of each lane's call as it runs in
        this schedule: the same round-robin steps again, reading the events
        captured in each lane's graph after every round."""
        acc = [[0.0] * 4 for _ in lns]
        for _ in range(rounds):
            e0.record(stream)
            run_steps(len(lns), lns)
            for a, ln in zip(acc, lns):
                for i, v in enumerate(hoph.hoph_plan_peek_timing(ln["plan"].handle)):
                    a[i] += v
        return [[v / rounds for v in a] for a in acc]

    # one batch at a time (lane 0 alone), then all lanes in flight
    ms1, clk1 = timed(lanes[:1])
    reps = min(args.steps, 200)
    ph1 = phases(lanes[:1], reps)[0]
    n_in = len(lanes)
    msn = clkn = phn = None
    if n_in > 1:
        msn, clkn = timed(lanes)
        phn = phases(lanes, max(1, reps // n_in))
    for ln in lanes:
        hoph.hoph_plan_enable_timing(ln["plan"].handle, False)

    world = int(os.environ.get("WORLD_SIZE", 1))
    pairs_per_step = nq * args.rows
    ms, clk = (msn, clkn) if msn is not None else (ms1, clk1)
    value = pairs_per_step * world * args.steps / (ms / 1e3)
    filt = ph1[1]
    # the streaming pass reads the first plane and the query sketches once
    alg_bytes = int(args.rows * KG * 4 + nq * KG * 4)
    traffic = NCU_TRAFFIC.get(filter_src_sha())
    roofline = {"bound": "hbm", "kernel": "filter_kernel",
                "achieved": alg_bytes / (filt / 1e3) / 1e9, "unit": "GB/s", "traffic": traffic,
                "alg_bytes": alg_bytes, "kernel_ms": filt}
    out = {"value": value, "ms": ms, "clocks": clk, "roofline": roofline,
           "gpu_launches": int(launches_per_step * args.steps),
           "schedule": ("%d batches in flight (a plan, stream, query batch and step graph per "
                        "lane; steps dealt round-robin)" % n_in if msn is not None
                        else "one batch at a time (graph replays)"),
           "decision_threshold": "%d/%d" % thr,
           "serial": {"ms_per_step": ms1 / args.steps,
                      "value": pairs_per_step * world * args.steps / (ms1 / 1e3),
                      "clocks": clk1, "phases_ms": dict(zip(PHASES, ph1))},
           "in_flight_phases_ms_by_lane": ([dict(zip(PHASES, p)) for p in phn] if phn else None),
           "autotune": {"best": best, "ms_by_candidate": tune_ms},
           "accepted_by_lane": [ln["n"] for ln in lanes],
           "stats": {"accepted": int(l0["n"]),
                     "survivors_entering_group": list(stats.entering[:4]),
                     "accepted_per_group": list(stats.accepted[:4]),
                     "rejected_per_group": list(stats.rejected[:4]),
                     "join_hits": int(stats.join_hits), "strategy": int(stats.strategy),
                     "rows_counted": int(stats.rows_counted)},
           "pairs": l0["pairs"]}
    knobs_used = dict(l0["plan"].exec_kwargs)
    for ln in lanes:
        ln["plan"].close()
    if truth_threshold_too and thr != T:
        # the same schedule and knobs at the ground-truth threshold itself
        out["value_at_T"] = headline_leg(args, planes, batches, dev, stream, T, barrier,
                                         max_over_ranks, local, knobs=knobs_used,
                                         truth_threshold_too=False)["value"]
    return out


PHASES = ("join_index", "filter", "count_candidates", "sort_stats")


def e2e_leg(args, thr, batches, planes, dev, world=1, sync=None, window=4096):
    """The step end to end through the public API from pinned host buffers,
    with the headline's lanes in flight: each lane (its own plan, stream and
    query batch) copies its sets in (H2D), sketches and queries them and
    copies the count and the first `window` pairs back (D2H); a lane's
    results are read (the rest of its pairs copied if there are more) before
    it takes its next batch.  Host wall time over --e2e-steps steps.  On
    several ranks every rank runs it between barriers (`sync(x)`: barrier
    and max over ranks of x) and the value counts all ranks' pairs."""
    import torch
    from paper_1805_11254_gb300 import hoph
    nq = args.queries
    cap = CAP
    lanes = []
    for b in batches:
        p = hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=thr, epsilon=EPS)
        h_ids = torch.from_numpy(np.ascontiguousarray(b["q_ids"]).view(np.int32)).pin_memory()
        h_off = torch.from_numpy(np.ascontiguousarray(b["q_off"])).pin_memory()
        lanes.append(dict(
            plan=p, s=torch.cuda.Stream(device=dev), h_ids=h_ids, h_off=h_off,
            d_ids=torch.empty_like(h_ids, device=dev), d_off=torch.empty_like(h_off, device=dev),
            q=torch.empty((p.G, nq, KG), dtype=torch.int32, device=dev),
            out=torch.empty((cap, 2), dtype=torch.int64, device=dev),
            cnt=torch.zeros(1, dtype=torch.int64, device=dev),
            h_cnt=torch.zeros(1, dtype=torch.int64).pin_memory(),
            h_out=torch.empty((cap, 2), dtype=torch.int64).pin_memory(),
            ev=torch.cuda.Event(), busy=False, h2d=0, d2h=0, pairs=0))
    n_lanes = len(lanes)

    def issue(ln):
        s = ln["s"]
        with torch.cuda.stream(s):
            ln["d_ids"].copy_(ln["h_ids"], non_blocking=True)
            ln["d_off"].copy_(ln["h_off"], non_blocking=True)
            hoph.oph_build_sketches(ln["plan"].handle, ln["d_ids"], ln["d_off"], nq, ln["q"], s)
            hoph.hoph_query_batch(ln["plan"].handle, hoph.HOPH_MODE_HOPH, ln["q"], nq, planes,
                                  args.rows, ln["out"], cap, ln["cnt"], None, s)
            ln["h_cnt"].copy_(ln["cnt"], non_blocking=True)
            ln["h_out"][:window].copy_(ln["out"][:window], non_blocking=True)
            ln["ev"].record(s)
        ln["h2d"] += ln["h_ids"].numel() * 4 + ln["h_off"].numel() * 8
        ln["d2h"] += 8 + 16 * window
        ln["busy"] = True

    def finish(ln):
        ln["ev"].synchronize()
        n = min(int(ln["h_cnt"][0]), cap)
        if n > window:  # the rest of the pairs
            ln["h_out"][window:n].copy_(ln["out"][window:n])
            ln["d2h"] += 16 * (n - window)
        ln["pairs"] = n
        ln["busy"] = False

    def run(k):
        for i in range(k):
            ln = lanes[i % n_lanes]
            if ln["busy"]:
                finish(ln)
            issue(ln)
        for ln in lanes:
            if ln["busy"]:
                finish(ln)
    sync = sync or (lambda x: x)
    run(3 * n_lanes)
    for ln in lanes:
        ln["h2d"] = ln["d2h"] = 0
    sync(0.0)
    t0 = time.perf_counter()
    run(args.e2e_steps)
    dt = sync((time.perf_counter() - t0) / args.e2e_steps)
    for ln in lanes:
        ln["plan"].check()
        ln["plan"].close()
    return {"value": nq * args.rows * world / dt, "unit": UNIT, "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": int(sum(ln["h2d"] for ln in lanes) / args.e2e_steps),
            "d2h_bytes_per_step": int(sum(ln["d2h"] for ln in lanes) / args.e2e_steps),
            "schedule": "%d batches in flight (one plan, stream and query batch each)" % n_lanes,
            "accepted_by_lane": [ln["pairs"] for ln in lanes],
            "path": "pinned host sets -> oph_build_sketches -> hoph_query_batch -> host pairs"}


EQUAL_RECALL_EPS = (1e-4, 1e-5, 1e-6, 1e-8, 0.0)
EQUAL_RECALL_T = ((699, 1000), (698, 1000), (697, 1000), (696, 1000), (695, 1000), (69, 100),
                  (68, 100), (67, 100))
RECALL_QUERIES = 4096


def recall_queries(off, coll_seed):
    """A larger query set for comparing recalls: 4,096 query sets, half of
    them planted near duplicates (J ~ U[0.6, 0.95]) of collection rows."""
    from paper_1805_11254_gb300 import synth
    return synth.query_batch(RECALL_QUERIES, 0.5, D, coll_seed, off, 0.6, 0.95, Q_SEED + 50,
                             PLANT_SEED + 50)


def eps_variants(args, planes, dq_ids, dq_off, nq, dev, stream, rq, reps=20,
                 variants=None):
    """The same step (sketch the query sets, HOPH query) at smaller error
    tolerances (or, with `variants` = [(thr, eps)], at other decision
    thresholds): the sketches do not depend on eps or the threshold, only the
    decisions do.  Returns {key: {"pairs", "ms"}} (key eps, or thr with
    variants): the pairs of the recall query set `rq` (one call of 4,096
    queries) and the eager CUDA-event time of the benchmark's 1,024-query
    step."""
    import torch
    from paper_1805_11254_gb300 import hoph
    rq_ids, rq_off = to_dev(rq["q_ids"], dev), to_dev(rq["q_off"], dev)
    n_rq = len(rq["q_off"]) - 1
    out = {}
    cap = CAP
    o = torch.empty((cap, 2), dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    runs = variants if variants is not None else [(T, e) for e in EQUAL_RECALL_EPS]
    for thr, eps in runs:
        key = thr if variants is not None else eps
        with hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=thr, epsilon=eps) as p:
            qp = torch.empty((p.G, nq, KG), dtype=torch.int32, device=dev)

            def step():
                hoph.oph_build_sketches(p.handle, dq_ids, dq_off, nq, qp, stream)
                hoph.hoph_query_batch(p.handle, hoph.HOPH_MODE_HOPH, qp, nq, planes, args.rows, o,
                                      cap, cnt, None, stream)
            for _ in range(3):
                step()
            p.check(stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            p.check(stream)
            ms = e0.elapsed_time(e1) / reps
            rqp = p.sketch(rq_ids, rq_off, n_rq, stream=stream)
            hoph.hoph_query_batch(p.handle, hoph.HOPH_MODE_HOPH, rqp, n_rq, planes, args.rows, o,
                                  cap, cnt, None, stream)
            p.check(stream)
            n = int(cnt.item())
            out[key] = {"pairs": o[:min(n, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
                        .copy(), "ms": ms}
    return out


def equal_recall(q, eps_runs, nq, rows, n_rq, thr_runs=None):
    """The largest eps at which HOPH's recall on the recall query set reaches
    plain OPH's, with the benchmark step's eager throughput at each eps.  The
    recall gap is the final estimator's (Lemma 3 weighs the groups by their
    space; OPH pools all bins), which no eps closes; so the largest decision
    threshold T' <= T at which HOPH (eps = 1e-4) reaches OPH's recall, ground
    truth still exact Jaccard >= T, is reported too."""
    target = q["oph_full_scan"]["recall"]
    pts = []
    for eps, r in eps_runs.items():
        m = q["hoph_eps_%g" % eps]
        pts.append({"eps": eps, "recall": m["recall"], "precision": m["precision"],
                    "ms_per_step_eager": r["ms"], "value": nq * rows / (r["ms"] / 1e3)})
    ok = [p for p in pts if p["recall"] >= target]
    best = max(ok, key=lambda p: p["eps"]) if ok else None
    tpts = []
    for thr, r in (thr_runs or {}).items():
        m = q["hoph_T_%d_%d" % thr]
        tpts.append({"T": "%d/%d" % thr, "t": thr[0] / thr[1], "recall": m["recall"],
                     "precision": m["precision"], "ms_per_step_eager": r["ms"],
                     "value": nq * rows / (r["ms"] / 1e3)})
    tok = [p for p in tpts if p["recall"] >= target]
    tbest = max(tok, key=lambda p: p["t"]) if tok else None
    return {"oph_full_scan_recall": target,
            "oph_full_scan_precision": q["oph_full_scan"]["precision"], "points": pts,
            "eps_at_equal_recall": best["eps"] if best else None,
            "value_at_equal_recall": best["value"] if best else None,
            "threshold_points": tpts,
            "decision_threshold_at_equal_recall": tbest["T"] if tbest else None,
            "precision_at_equal_recall": tbest["precision"] if tbest else None,
            "value_at_equal_recall_by_threshold": tbest["value"] if tbest else None,
            "unit": UNIT, "recall_queries": n_rq, "truly_similar": q["truly_similar"],
            "how": "recall of %d query sets (half planted) against exact Jaccard; eps only "
                   "changes the decisions; throughput = eager step timing (sketch + query) of "
                   "the 1,024-query step, not the graph replay" % n_rq}


def quality(qw, pairs_by_method, off, coll_seed, args, n_random_rows=2000):
    """Recall and precision against exact Jaccard >= T, per method, over one
    ground truth: every planted pair (known source) and every pair any method
    reported, with exact Jaccard from the CPU oracle.  A random sample of
    other (query, row) pairs bounds what all methods missed."""
    from oracle import oracle_c as oc
    from paper_1805_11254_gb300 import synth
    reps = {m: {(int(p["query"]), int(p["row"])) for p in ps} for m, ps in pairs_by_method.items()}
    planted = {(int(q), int(r)) for q, r in enumerate(qw["src"]) if r >= 0}
    rng = np.random.default_rng(Q_SEED + 99)
    n_rows = len(off) - 1
    rand_rows = rng.choice(n_rows, size=min(n_random_rows, n_rows), replace=False)
    nq = len(qw["q_off"]) - 1
    rand = {(q, int(r)) for q in range(nq) for r in rand_rows}
    cand = sorted(set().union(*reps.values()) | planted | rand)
    rows = sorted({r for _, r in cand})
    sets = [synth.counter_ids(coll_seed, int(off[r]), int(off[r + 1] - off[r]), D) for r in rows]
    c_ids, c_off = synth.pack_sets(sets)
    ridx = {r: i for i, r in enumerate(rows)}
    pa = np.asarray([q for q, _ in cand], dtype=np.int64)
    pb = np.asarray([ridx[r] for _, r in cand], dtype=np.int64)
    inter, uni = oc.jaccard_pairs(qw["q_ids"], qw["q_off"], c_ids, c_off, pa, pb)
    truth = {c for c, i, u in zip(cand, inter, uni) if u and i * T[1] >= T[0] * u}
    out = {}
    for m, rep in reps.items():
        tp = len(rep & truth)
        out[m] = {"reported": len(rep), "precision": tp / len(rep) if rep else 1.0,
                  "recall": tp / len(truth) if truth else 1.0}
    out["truly_similar"] = len(truth)
    out["random_pairs_checked"] = len(rand)
    out["truly_similar_among_random"] = len(truth & rand)
    out["ground_truth"] = ("exact Jaccard (CPU oracle) of planted pairs, of every pair either "
                           "method reported, and of %d random (query, row) pairs" % len(rand))
    return out


def sketch_leg(dev, stream, peaks, n_sets=1_000_000, steps=20):
    """Batched OPH sketching: 10^6 sets, lognormal sizes, Zipf(1.1) IDs over
    2^20, k = 256 (one plane)."""
    import torch
    from paper_1805_11254_gb300 import hoph, synth
    sizes = synth.lognormal_sizes(n_sets, 300, 1.0, 10, 20000, SKETCH_SEED)
    off = synth.offsets_from_sizes(sizes)
    n_ids = int(off[-1])
    cdf = synth.zipf_cdf(D, 1.1)
    d_cdf = torch.from_numpy(cdf).to(dev)
    d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
    hoph.hoph_synth_ids(SKETCH_SEED, 0, n_ids, D, 1, d_cdf, len(cdf), d_ids)
    d_off = to_dev(off, dev)
    from paper_1805_11254_gb300 import autotune
    with hoph.Plan(D, K, K, seed=PERM_SEED, thr=T, epsilon=EPS) as plan:
        out = torch.empty((1, n_sets, K), dtype=torch.int32, device=dev)
        for _ in range(3):
            plan.sketch(d_ids, d_off, n_sets, out=out, stream=stream)
        plan.check()
        best, tune_ms = autotune.tune_sketch(plan, d_ids, d_off, n_sets, out, stream)
        for _ in range(2):
            plan.sketch(d_ids, d_off, n_sets, out=out, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.sketch(d_ids, d_off, n_sets, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1) / steps
    bytes_ = 4 * n_ids + 8 * (n_sets + 1) + 4 * K * n_sets
    gbs = bytes_ / (ms / 1e3) / 1e9
    return {"sets_per_s": n_sets / (ms / 1e3), "ms_per_launch": ms,
            "autotune": {"sketch_cta_bits": best, "ms_by_bits": tune_ms},
            "workload": "1,000,000 sets, lognormal(300, 1.0) [10, 20000], Zipf(1.1) IDs over 2^20,"
                        " k = 256 OPH",
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / peaks["hbm_gbs"],
                         "traffic": NCU_TRAFFIC_SKETCH.get(sketch_src_sha()),
                         "algorithmic_bytes_per_launch": bytes_,
                         "binding_limit": "L1 data pipe: one random psi gather and one shared "
                                          "atomicMin per ID (IDs below 32 as bits), 76% of its "
                                          "peak in an ncu capture of this workload; DRAM moves "
                                          "about the algorithmic bytes"}}


def profile_shingle(args, dev, stream, reps=2):
    """The shingle regime's two sketches for ncu: --shingle-rows collection
    sets generated and sketched in the kernel (hoph_synth_sketch), then
    --shingle-queries stored query sets sketched, each `reps` times."""
    import torch
    from paper_1805_11254_gb300 import hoph, synth
    D4, K4, KG4, AB4 = 1 << 32, 512, 128, (2, 1)
    with hoph.Plan(D4, K4, KG4, *AB4, perm_kind=hoph.HOPH_PERM_HASH61, seed=PERM_SEED, thr=T,
                   epsilon=EPS) as plan:
        c_off = synth.offsets_from_sizes(synth.uniform_sizes(args.shingle_rows, 1000, 100000, 31))
        d_coff = to_dev(c_off, dev)
        planes = torch.empty((plan.G, args.shingle_rows, KG4), dtype=torch.int32, device=dev)
        for _ in range(reps):
            hoph.hoph_synth_sketch(plan.handle, 31, D4, d_coff, args.shingle_rows, planes, stream)
        q_off = synth.offsets_from_sizes(synth.uniform_sizes(args.shingle_queries, 1000, 100000,
                                                             34))
        d_qids = torch.empty(int(q_off[-1]), dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(35, 0, int(q_off[-1]), D4, 0, None, 0, d_qids, stream)
        qp = torch.empty((plan.G, args.shingle_queries, KG4), dtype=torch.int32, device=dev)
        for _ in range(reps):
            plan.sketch(d_qids, to_dev(q_off, dev), args.shingle_queries, out=qp, stream=stream)
        plan.check(stream)
        print(json.dumps({"profiled": "shingle", "collection_ids": int(c_off[-1]),
                          "query_ids": int(q_off[-1])}), flush=True)


def profile_self_join(args, off, coll_seed, dev, stream, batch=1536):
    """One hoph_self_join over the collection's first --rows rows ((1:2)HOPH,
    blocks of 1,536 rows, the library's default blocks in flight), for an ncu
    launch list; with --profile-compact over compact 16-bit planes
    (hoph_self_join16)."""
    import torch
    from paper_1805_11254_gb300 import hoph
    n = args.rows
    with hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=T, epsilon=EPS) as plan:
        n_ids = int(off[n])
        d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(coll_seed, 0, n_ids, D, 0, None, 0, d_ids)
        sketch = plan.sketch16 if args.profile_compact else plan.sketch
        planes = sketch(d_ids, to_dev(off[:n + 1], dev), n, stream=stream)
        del d_ids
        pairs, m, _ = plan.self_join("hoph", planes, n, batch=batch, stream=stream)
        print(json.dumps({"self_join_rows": n, "batch": batch, "accepted": m,
                          "compact": bool(args.profile_compact)}), flush=True)


def profile_oph1(args, off, coll_seed, dev, stream, launches=3):
    """One-query OPH full-scan launches for ncu: the strategy and knobs are
    tuned first as in the baseline leg, then the profiled launches run inside
    the NVTX range "oph1"."""
    import torch
    from paper_1805_11254_gb300 import autotune, hoph
    n_ids = int(off[-1])
    qw = query_sets(8, off, coll_seed)
    with hoph.Plan(D, K, K, seed=PERM_SEED, thr=T, epsilon=EPS) as plan:
        d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(coll_seed, 0, n_ids, D, 0, None, 0, d_ids)
        planes = plan.sketch(d_ids, to_dev(off, dev), args.rows)
        del d_ids
        q = plan.sketch(to_dev(qw["q_ids"], dev), to_dev(qw["q_off"], dev), 8)
        plan.check()
        cap = 1 << 12
        out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        qs = [q[:, i:i + 1].contiguous() for i in range(launches)]
        best, _ = autotune.tune_query(plan, hoph.HOPH_MODE_OPH_FULL, qs[0], 1, planes, args.rows,
                                      out, cap, cnt, stream,
                                      candidates=autotune.JOIN_CANDIDATES + autotune.DENSE_CANDIDATES)
        print(json.dumps({"tuned": best}), flush=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("oph1")
        for qp in qs:
            hoph.hoph_query_batch(plan.handle, hoph.HOPH_MODE_OPH_FULL, qp, 1, planes, args.rows,
                                  out, cap, cnt, None, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        plan.check()


def oph_baseline_leg(args, off, coll_seed, qw, dev, stream, hoph_value, rq, n_launch=8):
    """Plain OPH over all 256 bins (Eq. 6) on a uniform-OPH sketch of the same
    collection: the whole query batch in one call (the library picks the
    strategy), and one query per launch with the strategy (dense scan or
    value join) and knobs tuned for a single query.  Returns (leg, batched pairs,
    pairs of the recall query set rq)."""
    import torch
    from paper_1805_11254_gb300 import autotune, hoph
    n_ids = int(off[-1])
    with hoph.Plan(D, K, K, seed=PERM_SEED, thr=T, epsilon=EPS) as plan:
        d_off = to_dev(off, dev)
        d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(coll_seed, 0, n_ids, D, 0, None, 0, d_ids)
        planes = plan.sketch(d_ids, d_off, args.rows)
        del d_ids
        torch.cuda.empty_cache()
        dq_ids = to_dev(qw["q_ids"], dev)
        dq_off = to_dev(qw["q_off"], dev)
        nq = len(qw["q_off"]) - 1
        q_planes = plan.sketch(dq_ids, dq_off, nq)
        plan.check()
        cap = 1 << 16
        out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(hoph.STATS_WORDS, dtype=torch.int64, device=dev)

        # the whole batch in one call
        plan.set_exec()
        hoph.hoph_query_batch(plan.handle, hoph.HOPH_MODE_OPH_FULL, q_planes, nq, planes,
                              args.rows, out, cap, cnt, st, stream)
        plan.check(stream)
        n_b = int(cnt.item())
        pairs_b = out[:min(n_b, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1).copy()
        strategy_b = int(hoph.hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes()).strategy)
        n_rq = len(rq["q_off"]) - 1
        rqp = plan.sketch(to_dev(rq["q_ids"], dev), to_dev(rq["q_off"], dev), n_rq)
        hoph.hoph_query_batch(plan.handle, hoph.HOPH_MODE_OPH_FULL, rqp, n_rq, planes, args.rows,
                              out, cap, cnt, None, stream)
        plan.check(stream)
        n_r = int(cnt.item())
        pairs_rq = out[:min(n_r, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1).copy()
        del rqp
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            hoph.hoph_query_batch(plan.handle, hoph.HOPH_MODE_OPH_FULL, q_planes, nq, planes,
                                  args.rows, out, cap, cnt, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1) / reps

        # one query per launch, the strategy and knobs tuned for Q = 1
        planted = [q for q in range(nq) if qw["src"][q] >= 0][:n_launch]
        qs = [q_planes[:, q:q + 1].contiguous() for q in planted]
        best, tune_ms = autotune.tune_query(plan, hoph.HOPH_MODE_OPH_FULL, qs[0], 1, planes,
                                            args.rows, out, cap, cnt, stream,
                                            candidates=autotune.JOIN_CANDIDATES + autotune.DENSE_CANDIDATES)
        for qp in qs[:2]:
            hoph.hoph_query_batch(plan.handle, hoph.HOPH_MODE_OPH_FULL, qp, 1, planes, args.rows,
                                  out, cap, cnt, None, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for qp in qs:
            hoph.hoph_query_batch(plan.handle, hoph.HOPH_MODE_OPH_FULL, qp, 1, planes, args.rows,
                                  out, cap, cnt, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1) / len(qs)
        del planes
        torch.cuda.empty_cache()
    v = args.rows / (ms / 1e3)
    plane_bytes = args.rows * K * 4
    leg = {"value": v, "unit": UNIT, "ms_per_query_launch": ms,
           "hbm_GB_per_s": plane_bytes / (ms / 1e3) / 1e9,
           "hoph_speedup": hoph_value / v,
           "tuned": best, "tune_ms_by_candidate": tune_ms,
           "how": "mode OPH_FULL over all 256 bins (10.24 GB of planes per launch), one query "
                  "per launch, %d launches, strategy and knobs tuned for one query" % len(qs),
           "batched": {"value": nq * args.rows / (ms_b / 1e3), "unit": UNIT, "ms_per_batch": ms_b,
                       "queries": nq, "strategy": strategy_b, "accepted": n_b,
                       "hoph_speedup": hoph_value / (nq * args.rows / (ms_b / 1e3))}}
    return leg, pairs_b, pairs_rq


def serving_leg(args, planes, dev, oph_leg):
    """Continuous batching against the resident collection: Poisson arrivals
    of requests of U[1, 256] query sets (lognormal sizes, median 300); each
    batch (<= 1,024 sets) replays one captured graph.  p50/p99 latency from
    arrival to results on the host, and throughput, per arrival rate."""
    from paper_1805_11254_gb300 import serve, synth
    plan_kw = dict(D=D, k=K, k_group=KG, a=AB[0], b=AB[1], seed=PERM_SEED, thr=T, epsilon=EPS)
    buckets = (64, 256, 1024)
    id_cap = 4 << 20
    ctr = [0]

    def sets_for(rng, n):
        sizes = synth.lognormal_sizes(n, 300, 1.0, 10, 20000, int(rng.integers(1 << 31)))
        out = []
        for sz in sizes:
            out.append(synth.counter_ids(977, ctr[0], int(sz), D))
            ctr[0] += int(sz)
        return out

    by_streams = {}
    for n_streams in (2, 4):
        ex = serve.GpuExecutor(plan_kw, planes, args.rows, "hoph", buckets, None,
                               n_streams=n_streams, max_ids=id_cap)
        results = []
        try:
            for i, rate in enumerate(float(x) for x in args.serve_rates.split(",")):
                reqs = serve.poisson_requests(rate, args.serve_seconds, 100 + i, sets_for)
                t0 = time.perf_counter()
                done = serve.serve(ex, serve.Batcher(buckets, ex.id_capacity), reqs)
                wall = time.perf_counter() - t0
                ok = [r for r in done if r.error is None]
                n_sets = sum(len(r.sets) for r in ok)
                summ = serve.latency_summary(ok)
                summ.update({"rate_query_sets_per_s": rate, "query_sets": n_sets,
                             "throughput_query_sets_per_s": n_sets / wall,
                             "pair_comparisons_per_s": n_sets * args.rows / wall,
                             "rejected": len(done) - len(ok)})
                results.append(summ)
        finally:
            ex.close()
        by_streams[n_streams] = {"id_capacity_per_batch": ex.id_capacity, "rates": results}
    return {"rates": by_streams[4]["rates"], "rates_by_streams": by_streams,
            "collection_rows": args.rows, "batch_slots": list(buckets),
            "one_request_per_launch_oph_capacity_query_sets_per_s":
                1e3 / oph_leg["ms_per_query_launch"],
            "how": "2 or 4 streams x 1 plan each, one CUDA graph per (stream, batch size); H2D "
                   "of a batch's sets and its sketching overlap other streams' queries; IDs per "
                   "batch sized from the free HBM at start (75%, split over the streams, at "
                   "most 4M)"}


def compact_leg(args, off, coll_seed, dq_ids, dq_off, nq, pairs_ref, dev, stream, peaks, thr,
                steps=200):
    """The benchmark step over compact planes: every bin of the (1:2) layout
    over 2^20 is at most 5,462 values wide, so the stored offsets fit in 16
    bits (oph_build_sketches16 / hoph_query_batch16) and the streamed plane
    halves.  Same pairs as the uint32 planes (checked), timed as a graph."""
    import torch
    from paper_1805_11254_gb300 import hoph
    plan = hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=thr, epsilon=EPS)
    n_ids = int(off[-1])
    d_off = to_dev(off, dev)
    d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
    hoph.hoph_synth_ids(coll_seed, 0, n_ids, D, 0, None, 0, d_ids)
    c16 = plan.sketch16(d_ids, d_off, args.rows)
    plan.check()
    del d_ids
    torch.cuda.empty_cache()
    q16 = torch.empty((plan.G, nq, KG), dtype=torch.int16, device=dev)
    cap = CAP
    out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)

    def step(s):
        hoph.oph_build_sketches16(plan.handle, dq_ids, dq_off, nq, q16, s)
        hoph.hoph_query_batch16(plan.handle, hoph.HOPH_MODE_HOPH, q16, nq, c16, args.rows, out,
                                cap, cnt, None, s)
    from paper_1805_11254_gb300 import autotune
    hoph.oph_build_sketches16(plan.handle, dq_ids, dq_off, nq, q16, stream)
    best, tune_ms = autotune.tune_query(plan, hoph.HOPH_MODE_HOPH, q16, nq, c16, args.rows, out,
                                        cap, cnt, stream)
    for _ in range(3):
        step(stream)
    plan.check(stream)
    n = int(cnt.item())
    got = out[:min(n, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
    same = bool(n == len(pairs_ref) and np.array_equal(got, pairs_ref))
    hoph.hoph_plan_enable_timing(plan.handle, True)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            step(side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(torch.cuda.current_stream())
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    phase = [0.0] * 4
    for _ in range(steps):
        graph.replay()
        phase = [a + b for a, b in zip(phase, hoph.hoph_plan_peek_timing(plan.handle))]
    filt = phase[1] / steps
    plan.check()
    hoph.hoph_plan_enable_timing(plan.handle, False)
    # batches in flight (two to four), as for the uint32 headline
    lanes = [dict(plan=plan, q=q16, out=out, cnt=cnt)]
    for _ in range(3):
        p2 = hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=thr, epsilon=EPS)
        p2.set_exec(**plan.exec_kwargs)
        lanes.append(dict(plan=p2, q=torch.empty_like(q16), out=torch.empty_like(out),
                          cnt=torch.zeros_like(cnt)))

    def lane_step(ln, s):
        hoph.oph_build_sketches16(ln["plan"].handle, dq_ids, dq_off, nq, ln["q"], s)
        hoph.hoph_query_batch16(ln["plan"].handle, hoph.HOPH_MODE_HOPH, ln["q"], nq, c16,
                                args.rows, ln["out"], cap, ln["cnt"], None, s)
    for ln in lanes[1:]:
        for _ in range(3):
            lane_step(ln, stream)
    torch.cuda.synchronize()
    ms_in_flight = {}
    for n_in in (2, 3, 4):
        streams = [torch.cuda.Stream(device=dev) for _ in range(n_in)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream()
            for st_, ln in zip(streams, lanes):
                st_.wait_stream(cs)
                lane_step(ln, st_)
            for st_ in streams:
                cs.wait_stream(st_)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps // n_in):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_in_flight[n_in] = e0.elapsed_time(e1) / (n_in * (steps // n_in))
    for ln in lanes:
        ln["plan"].check()
    for ln in lanes[1:]:
        ln["plan"].close()
    ms2 = min(ms_in_flight.values())
    plan.close()
    del c16
    torch.cuda.empty_cache()
    alg = int(args.rows * KG * 2 + nq * KG * 2)
    ach = alg / (filt / 1e3) / 1e9
    ms_serial = ms
    ms = min(ms, ms2)
    # lanes_per_row 0 is the library's choice: the striped filter for 16-bit planes
    striped = best is None or (best.get("strategy", 1) != 0 and
                               best.get("lanes_per_row", 0) in (0, 32))
    return {"value": nq * args.rows / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "ms_per_step_one_batch_at_a_time": ms_serial,
            "ms_per_step_by_batches_in_flight": ms_in_flight,
            "same_pairs_as_uint32_planes": same, "plane_bytes": args.rows * K * 2,
            "autotune": {"best": best, "ms_by_candidate": tune_ms},
            "roofline": {"bound": "hbm",
                         "kernel": ("filter_striped_kernel" if striped else "filter_kernel")
                         + " (uint16 planes)",
                         "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"], "algorithmic_bytes_per_launch": alg,
                         "kernel_ms_per_launch": filt,
                         "traffic": NCU_TRAFFIC_STRIPED.get(filter_src_sha(True))
                         if striped else None},
            "how": "same collection and query sets; sketch values stored as 16-bit bin offsets "
                   "(empty = 0xFFFF); CUDA graph replays, CUDA events"}


def self_join_leg(off, coll_seed, dev, stream, n_base=1_000_000, n_planted=1000,
                  batches=(1024, 1536, 2048), lanes=(3, 4, 6, 8), reps=3):
    """All near-duplicate pairs inside one collection (hoph_self_join): the
    first 10^6 rows of the query workload's collection plus 1,000 planted
    near duplicates of random rows among them (J ~ U[0.6, 0.95]), (1:2)HOPH;
    the rows taken as queries per block and the blocks in flight are chosen
    by timing (both are execution choices; the result is checked to be the
    same for every choice).  Reports pairs compared per second and how many
    planted pairs with exact Jaccard >= T were found."""
    import torch
    from oracle import oracle_c as oc
    from paper_1805_11254_gb300 import hoph, synth
    rng = np.random.default_rng(PLANT_SEED + 7)
    src = np.sort(rng.choice(n_base, n_planted, replace=False))
    bases = [synth.counter_ids(coll_seed, int(off[r]), int(off[r + 1] - off[r]), D) for r in src]
    planted, _ = synth.plant_near_duplicates(bases, D, 0.6, 0.95, PLANT_SEED + 8)
    p_ids, p_off = synth.pack_sets(planted)
    b_ids, b_off = synth.pack_sets([np.unique(b) for b in bases])
    inter, uni = oc.jaccard_pairs(b_ids, b_off, p_ids, p_off, np.arange(n_planted),
                                  np.arange(n_planted))
    truly = inter * T[1] >= T[0] * uni
    n = n_base + n_planted
    with hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=T, epsilon=EPS) as plan:
        n_ids = int(off[n_base])
        d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(coll_seed, 0, n_ids, D, 0, None, 0, d_ids)
        base_planes = plan.sketch(d_ids, to_dev(off[:n_base + 1], dev), n_base)
        base16 = plan.sketch16(d_ids, to_dev(off[:n_base + 1], dev), n_base)
        del d_ids
        pl_planes = plan.sketch(to_dev(p_ids, dev), to_dev(p_off, dev), n_planted)
        pl16 = plan.sketch16(to_dev(p_ids, dev), to_dev(p_off, dev), n_planted)
        planes = torch.cat([base_planes, pl_planes], dim=1).contiguous()
        planes16 = torch.cat([base16, pl16], dim=1).contiguous()
        del base_planes, pl_planes, base16, pl16
        plan.check()
        cap = 1 << 20
        out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms_by_choice, ref = {}, None
        for b in batches:
            for ln in lanes:
                plan.update_exec(join_lanes=ln)
                hoph.hoph_self_join(plan.handle, hoph.HOPH_MODE_HOPH, planes, n, b, out, cap,
                                    cnt, None, stream)
                plan.check(stream)
                m = int(cnt.item())
                got = out[:min(m, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1).copy()
                if ref is None:
                    ref = got
                elif not np.array_equal(got, ref):
                    raise RuntimeError("the self-join's block size or lanes changed its result")
                e0.record(stream)
                for _ in range(reps):
                    hoph.hoph_self_join(plan.handle, hoph.HOPH_MODE_HOPH, planes, n, b, out, cap,
                                        cnt, None, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                plan.check(stream)
                ms_by_choice["%d rows x %d lanes" % (b, ln)] = e0.elapsed_time(e1) / reps
        best = min(ms_by_choice, key=ms_by_choice.get)
        ms = ms_by_choice[best]
        pairs = ref
        m = len(ref)
        del planes
        # the same self-join over compact 16-bit planes (hoph_self_join16:
        # the striped filter), the result checked against the uint32 one
        ms16_by_choice, same16 = {}, True
        for b in batches:
            for ln in lanes[-2:]:
                plan.update_exec(join_lanes=ln)
                hoph.hoph_self_join16(plan.handle, hoph.HOPH_MODE_HOPH, planes16, n, b, out, cap,
                                      cnt, None, stream)
                plan.check(stream)
                m16 = int(cnt.item())
                got = out[:min(m16, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
                same16 = same16 and bool(np.array_equal(got, ref))
                e0.record(stream)
                for _ in range(reps):
                    hoph.hoph_self_join16(plan.handle, hoph.HOPH_MODE_HOPH, planes16, n, b, out,
                                          cap, cnt, None, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                plan.check(stream)
                ms16_by_choice["%d rows x %d lanes" % (b, ln)] = e0.elapsed_time(e1) / reps
        best16 = min(ms16_by_choice, key=ms16_by_choice.get)
        # the same compact self-join split in two parts (hoph_self_join_part, as over
        # two GPUs each holding the collection): each part timed alone on this GPU
        b16, ln16 = (int(x) for x in best16.replace(" rows x", "").split()[:2])
        plan.update_exec(join_lanes=ln16)
        split_ms, split_pairs = [], []
        for part in range(2):
            hoph.hoph_self_join_part(plan.handle, hoph.HOPH_MODE_HOPH, planes16, n, b16, part, 2,
                                     out, cap, cnt, None, stream)
            plan.check(stream)
            mp = int(cnt.item())
            split_pairs.append(out[:min(mp, cap)].cpu().numpy().view(hoph.PAIR_DTYPE)
                               .reshape(-1).copy())
            e0.record(stream)
            for _ in range(reps):
                hoph.hoph_self_join_part(plan.handle, hoph.HOPH_MODE_HOPH, planes16, n, b16, part,
                                         2, out, cap, cnt, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            split_ms.append(e0.elapsed_time(e1) / reps)
        from paper_1805_11254_gb300 import shard
        split_same = bool(np.array_equal(shard.merge_pairs(split_pairs), ref))
        del planes16
        torch.cuda.empty_cache()
    found = {(int(p["query"]), int(p["row"])) for p in pairs}
    want = {(int(src[i]), n_base + i) for i in range(n_planted) if truly[i]}
    compared = n * (n - 1) // 2
    return {"rows": n, "pairs_compared": compared, "ms": ms,
            "value": compared / (ms / 1e3), "unit": UNIT, "accepted": m,
            "ms_by_block_rows_and_lanes": ms_by_choice,
            "planted_truly_similar": len(want), "planted_found": len(want & found),
            "compact": {"ms": ms16_by_choice[best16],
                        "value": compared / (ms16_by_choice[best16] / 1e3),
                        "same_pairs_as_uint32_planes": same16,
                        "ms_by_block_rows_and_lanes": ms16_by_choice,
                        "how": "hoph_self_join16 over compact 16-bit planes, blocks of %s"
                               % best16,
                        "split_in_two": {"ms_by_part": split_ms, "same_pairs": split_same,
                                         "how": "hoph_self_join_part, parts 0 and 1 of 2, "
                                                "each timed alone on this GPU"}},
            "how": "hoph_self_join, blocks of %s in flight, each block's rows as queries against "
                   "the rows from the block on; (1:2)HOPH k=256 k'=64, T=0.7, eps=1e-4" % best}


SWEEP_T = ((1, 2), (3, 5), (7, 10), (4, 5), (9, 10))
SWEEP_EPS = (1e-3, 1e-4, 1e-5)


def large_output_leg(dev, stream, reps=5):
    """A query whose output is over a million accepted pairs (1,200 x 1,100
    sketches over two values per bin, GOPH k = 64, k' = 32, T = 2/5, the
    case of the tests): the comparison's and the output sort's phase times
    from the library's CUDA events, with the capacity above the one-CTA
    sort's limit (many-CTA runs and merges)."""
    import torch
    from paper_1805_11254_gb300 import hoph
    rng = np.random.default_rng(77)
    Dl, k, kg, nq, nr = 1 << 16, 64, 32, 1200, 1100
    q_rows = rng.integers(0, 2, (nq, k)).astype(np.uint32)
    c_rows = rng.integers(0, 2, (nr, k)).astype(np.uint32)
    q_rows[rng.random((nq, k)) < 0.05] = hoph.HOPH_EMPTY_VALUE
    c_rows[rng.random((nr, k)) < 0.05] = hoph.HOPH_EMPTY_VALUE

    def planes(rows):
        p = np.ascontiguousarray(rows.reshape(len(rows), k // kg, kg).transpose(1, 0, 2))
        return to_dev(p, dev)
    q, c = planes(q_rows), planes(c_rows)
    cap = 1 << 21
    out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    with hoph.Plan(Dl, k, kg, seed=1, thr=(2, 5), epsilon=EPS) as plan:
        hoph.hoph_query_batch(plan.handle, "goph", q, nq, c, nr, out, cap, cnt, None, stream)
        plan.check(stream)
        n = int(cnt.item())
        got = out[:min(n, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
        key = got["query"].astype(np.int64) * nr + got["row"]
        ordered = bool(np.all(np.diff(key) > 0))
        hoph.hoph_plan_enable_timing(plan.handle, True)
        for _ in range(reps):
            hoph.hoph_query_batch(plan.handle, "goph", q, nq, c, nr, out, cap, cnt, None, stream)
        ph, calls, launches = hoph.hoph_plan_read_timing(plan.handle)
        hoph.hoph_plan_enable_timing(plan.handle, False)
        plan.check(stream)
    return {"accepted": n, "in_order": ordered, "capacity": cap,
            "compare_ms": (ph[0] + ph[1] + ph[2]) / max(calls, 1),
            "sort_ms": ph[3] / max(calls, 1), "launches_per_call": launches / max(calls, 1),
            "how": "GOPH, 1,200 queries x 1,100 rows, dense scan; sort = many-CTA run sort and "
                   "merge passes (16 B records)"}


def sweep_leg(dev, stream, reps=5):
    """Threshold and tolerance sweeps on the 5,000-set workload (D = 2^16,
    k = 128, 50 planted queries at J ~ U[0.3, 0.95]): MinWise (128
    permutations), plain OPH, GOPH (4 x 32) and (1:1)HOPH (k' = 32), each with
    recall and precision against exact Jaccard of all 250,000 pairs and the
    query time; T in 0.5..0.9 at eps = 1e-4, then eps in 1e-3..1e-5 at T = 0.7
    for the early-terminating methods."""
    import torch
    from oracle import oracle_c as oc
    from paper_1805_11254_gb300 import hoph, synth
    w = synth.small_parity_workload()
    Dw, k, kg, nq = w["D"], 128, 32, len(w["q_off"]) - 1
    n = len(w["off"]) - 1
    pa = np.repeat(np.arange(nq, dtype=np.int64), n)
    pb = np.tile(np.arange(n, dtype=np.int64), nq)
    inter, uni = oc.jaccard_pairs(w["q_ids"], w["q_off"], w["ids"], w["off"], pa, pb)
    inter = inter.reshape(nq, n)
    uni = uni.reshape(nq, n)
    d = {key: to_dev(w[key], dev) for key in ("ids", "off", "q_ids", "q_off")}
    layouts = {"minwise": (0, 0), "oph_full": (0, 0), "goph": (0, 0), "hoph_1_1": (1, 1)}
    modes = {"minwise": hoph.HOPH_MODE_MINWISE_FULL, "oph_full": hoph.HOPH_MODE_OPH_FULL,
             "goph": hoph.HOPH_MODE_GOPH, "hoph_1_1": hoph.HOPH_MODE_HOPH}
    sk, sketch_ms = {}, {}
    for m, ab in layouts.items():  # sketches depend on psi and the layout only
        with hoph.Plan(Dw, k, kg, *ab, seed=PERM_SEED, minwise_k=k if m == "minwise" else 0) as p:
            make = p.minwise if m == "minwise" else p.sketch
            sk[m] = (make(d["q_ids"], d["q_off"], nq), make(d["ids"], d["off"], n))
            p.check()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                make(d["ids"], d["off"], n, out=sk[m][1], stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            sketch_ms[m] = e0.elapsed_time(e1) / reps
    out = []
    cap = 1 << 16
    o = torch.empty((cap, 2), dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    settings = [(m, t, 1e-4) for t in SWEEP_T for m in layouts] + \
               [(m, (7, 10), e) for e in SWEEP_EPS for m in ("goph", "hoph_1_1")]
    for m, t, eps in settings:
        with hoph.Plan(Dw, k, kg, *layouts[m], seed=PERM_SEED, thr=t, epsilon=eps,
                       minwise_k=k if m == "minwise" else 0) as p:
            qs, cs = sk[m]
            hoph.hoph_query_batch(p.handle, modes[m], qs, nq, cs, n, o, cap, cnt, None, stream)
            p.check(stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                hoph.hoph_query_batch(p.handle, modes[m], qs, nq, cs, n, o, cap, cnt, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            p.check(stream)
            ms = e0.elapsed_time(e1) / reps
            c = int(cnt.item())
            pairs = o[:min(c, cap)].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
        truth = (uni > 0) & (inter * t[1] >= t[0] * uni)
        got = np.zeros_like(truth)
        got[pairs["query"].astype(np.int64), pairs["row"]] = True
        tp = int((got & truth).sum())
        out.append({"method": m, "T": "%d/%d" % t, "eps": eps, "ms": ms, "reported": int(got.sum()),
                    "truly_similar": int(truth.sum()),
                    "recall": tp / int(truth.sum()) if truth.any() else 1.0,
                    "precision": tp / int(got.sum()) if got.any() else 1.0})
    return {"workload": "5,000 sets of U[50, 500] distinct IDs over 2^16, 50 planted queries at "
                        "J ~ U[0.3, 0.95], k = 128 (GOPH 4 x 32, 1:1 HOPH k' = 32, MinWise 128 "
                        "permutations); ground truth: exact Jaccard of all 250,000 pairs",
            "collection_sketch_ms": sketch_ms, "points": out}


# Multiplies per ID on the hashed-psi sketch path (read off the kernels): the
# generator's SplitMix64 step (3 low 64-bit products) and its scaling to
# [0, D) (a 32-bit high half), psi = ((a x + b) mod 2^61-1) >> 29 (1 low + 1
# high 64-bit product), and the bin floor(o nb / z) by the region's magic
# multiplier (2 32-bit multiplies: a wide product and a high half)
ALU_MULS_GENERATED = {"lo": 4, "hi": 1, "imad32": 3}
ALU_MULS_STORED = {"lo": 1, "hi": 1, "imad32": 2}


def alu_peak_leg(dev, stream, target_ms=30.0):
    """Measured integer peaks (hoph_int_probe): 32-bit multiply-adds and the
    low and high halves of 64-bit products per second, each from a launch of
    about target_ms, with the SM clock sampled meanwhile."""
    import torch
    from paper_1805_11254_gb300 import hoph
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    threads = sms * 8 * 256
    sink = torch.empty(threads, dtype=torch.int64, device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = {}
    for kind, name in ((0, "imad32"), (1, "mul64_lo"), (2, "mul64_hi")):
        iters = 256
        for _ in range(12):  # grow until a launch takes about target_ms
            hoph.hoph_int_probe(kind, iters, sink, stream)
            e0.record(stream)
            hoph.hoph_int_probe(kind, iters, sink, stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if ms >= target_ms or iters >= 1 << 24:
                break
            iters = min(1 << 24, int(iters * max(2.0, target_ms / max(ms, 1e-3))))
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        time.sleep(0.2)
        e0.record(stream)
        for _ in range(3):
            hoph.hoph_int_probe(kind, iters, sink, stream)
        e1.record(stream)
        e1.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / 3
        ops = 8.0 * iters * threads
        rate = ops / (ms / 1e3)
        mhz = clk["sm_mhz"] if clk else None
        out[name] = {"ops_per_s": rate, "ms": ms, "iters": iters,
                     "per_sm_per_clock": rate / sms / (mhz * 1e6) if mhz else None,
                     "sm_mhz": mhz}
    return out


def alu_roofline(ids_per_s, muls, peak):
    """IDs/s against the IDs/s the measured multiply rates allow at `muls`
    64-bit low and high products and 32-bit multiplies per ID."""
    ideal = 1.0 / (muls["lo"] / peak["mul64_lo"]["ops_per_s"] +
                   muls["hi"] / peak["mul64_hi"]["ops_per_s"] +
                   muls.get("imad32", 0) / peak["imad32"]["ops_per_s"])
    return {"bound": "alu", "achieved": ids_per_s, "peak": ideal, "unit": "IDs/s",
            "frac": ids_per_s / ideal, "muls_per_id": muls,
            "peak_source": "measured (hoph_int_probe multiply rates, this run)"}


def shingle_leg(args, dev, stream, peaks, q_batch=1024, n_planted=32):
    """Large-set shingle regime: IDs uniform over 2^32, psi the 2-universal
    hash mod 2^61-1, (2:1)HOPH with k = 512, k' = 128 (G = 4), T = 0.7.  The
    collection (sizes U[1000, 100000]) is generated and sketched inside the
    kernel; the query sets (same law) are stored in HBM and sketched like any
    input; queries run in batches of 1,024 through the hashed join."""
    import torch
    from paper_1805_11254_gb300 import hoph, synth
    D4, K4, KG4, AB4 = 1 << 32, 512, 128, (2, 1)
    seed_c, seed_q = 31, 32
    out = {"workload": "collection %d sets and %d queries, sizes U[1000, 100000], IDs uniform "
                       "over 2^32, (2:1)HOPH k=512 k'=128, T=0.7, eps=1e-4"
                       % (args.shingle_rows, args.shingle_queries)}
    with hoph.Plan(D4, K4, KG4, *AB4, perm_kind=hoph.HOPH_PERM_HASH61, seed=PERM_SEED, thr=T,
                   epsilon=EPS) as plan:
        c_sizes = synth.uniform_sizes(args.shingle_rows, 1000, 100000, seed_c)
        c_off = synth.offsets_from_sizes(c_sizes)
        d_coff = to_dev(c_off, dev)
        planes = torch.empty((plan.G, args.shingle_rows, KG4), dtype=torch.int32, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hoph.hoph_synth_sketch(plan.handle, seed_c, D4, d_coff, args.shingle_rows, planes, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1)
        alu = alu_peak_leg(dev, stream)
        out["alu_peak"] = alu
        ids_s = int(c_off[-1]) / (ms / 1e3)
        out["collection_generate_and_sketch"] = {
            "sets_per_s": args.shingle_rows / (ms / 1e3), "ids_per_s": ids_s,
            "ms": ms, "ids": int(c_off[-1]),
            "roofline": alu_roofline(ids_s, ALU_MULS_GENERATED, alu)}
        # query sets: a few planted near duplicates of collection rows, the rest fresh
        rng = np.random.default_rng(seed_q)
        src = rng.integers(0, args.shingle_rows, n_planted)
        bases = [synth.counter_ids(seed_c, int(c_off[r]), int(c_sizes[r]), D4) for r in src]
        planted, _ = synth.plant_near_duplicates(bases, D4, 0.75, 0.98, seed_q + 1)
        p_ids, p_off = synth.pack_sets(planted)
        q_sizes = np.concatenate([np.diff(p_off),
                                  synth.uniform_sizes(args.shingle_queries - n_planted, 1000,
                                                      100000, seed_q + 2)])
        q_off = synth.offsets_from_sizes(q_sizes)
        d_qids = torch.empty(int(q_off[-1]), dtype=torch.int32, device=dev)
        d_qids[:len(p_ids)].copy_(torch.from_numpy(p_ids.view(np.int32)))
        hoph.hoph_synth_ids(seed_q + 3, 0, int(q_off[-1]) - len(p_ids), D4, 0, None, 0,
                            d_qids[len(p_ids):], stream)
        d_qoff = to_dev(q_off, dev)
        nq = args.shingle_queries
        q_planes = torch.empty((plan.G, nq, KG4), dtype=torch.int32, device=dev)
        for _ in range(2):
            plan.sketch(d_qids, d_qoff, nq, out=q_planes, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        reps = 3
        for _ in range(reps):
            plan.sketch(d_qids, d_qoff, nq, out=q_planes, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1) / reps
        byts = 4 * int(q_off[-1]) + 8 * (nq + 1) + 4 * K4 * nq
        gbs = byts / (ms / 1e3) / 1e9
        out["query_sketch"] = {"sets_per_s": nq / (ms / 1e3), "ms": ms, "ids": int(q_off[-1]),
                               "GB_per_s": gbs, "hbm_frac": gbs / peaks["hbm_gbs"],
                               "roofline": alu_roofline(int(q_off[-1]) / (ms / 1e3),
                                                        ALU_MULS_STORED, alu)}
        del d_qids
        # batches of 1,024 query sketches against the collection
        cap = 1 << 16
        outp = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(hoph.STATS_WORDS, dtype=torch.int64, device=dev)
        batches = [q_planes[:, b:b + q_batch].contiguous() for b in range(0, nq, q_batch)]
        sizes_b = [bq.shape[1] for bq in batches]
        from paper_1805_11254_gb300 import autotune
        best, tune_ms = autotune.tune_query(plan, hoph.HOPH_MODE_HOPH, batches[0], sizes_b[0],
                                            planes, args.shingle_rows, outp, cap, cnt, stream)
        hoph.hoph_query_batch(plan.handle, "hoph", batches[0], sizes_b[0], planes,
                              args.shingle_rows, outp, cap, cnt, st, stream)
        torch.cuda.synchronize()
        plan.check()
        first = outp[:int(cnt.item())].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
        found = {(int(p["query"]), int(p["row"])) for p in first}
        stats = hoph.hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes())
        e0.record(stream)
        for bq, n in zip(batches, sizes_b):
            hoph.hoph_query_batch(plan.handle, "hoph", bq, n, planes, args.shingle_rows, outp, cap,
                                  cnt, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1)
        plane_gb = args.shingle_rows * KG4 * 4 / 1e9
        out["hoph_query"] = {
            "pair_comparisons_per_s": nq * args.shingle_rows / (ms / 1e3),
            "ms_per_1024_batch": ms / len(batches), "batches": len(batches),
            "first_plane_GB_per_s": plane_gb / (ms / len(batches) / 1e3),
            "autotune": {"best": best, "ms_by_candidate": tune_ms},
            "strategy": int(stats.strategy), "candidate_rows_first_batch": int(stats.rows_counted),
            "planted_found": sum((q, int(r)) in found for q, r in enumerate(src)),
            "planted": n_planted}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
