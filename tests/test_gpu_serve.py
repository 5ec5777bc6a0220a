"""The continuous-batching service returns, for every request, the same
pairs whether the request was served alone or batched with others, and
those pairs are the oracle's."""
import numpy as np
import pytest

from gpu_helpers import device, planes_to_rows, to_dev, torch  # noqa: F401
from oracle import oracle_c as oc
from paper_1805_11254_gb300 import hoph, serve, synth

pytestmark = pytest.mark.gpu


def test_results_identical_alone_and_in_the_mix():
    dev = device()
    w = synth.small_parity_workload(n=4000, n_queries=120)
    D, k, kg, ab = w["D"], 128, 32, (1, 2)
    plan_kw = dict(D=D, k=k, k_group=kg, a=ab[0], b=ab[1], seed=1, thr=(7, 10), epsilon=1e-4)
    with hoph.Plan(**plan_kw) as plan:
        coll = plan.sketch(to_dev(w["ids"], dev), to_dev(w["off"], dev), 4000)
        plan.check()
    qsets = [w["q_ids"][w["q_off"][i]:w["q_off"][i + 1]] for i in range(120)]
    rng = np.random.default_rng(5)
    reqs, pos, rid = [], 0, 0
    while pos < 120:
        n = int(rng.integers(1, 9))
        reqs.append(serve.Request(rid, qsets[pos:pos + n], 0.0005 * rid))
        pos += n
        rid += 1
    ex = serve.GpuExecutor(plan_kw, coll, 4000, "hoph", (8, 32), 60000)
    try:
        mixed = serve.serve(ex, serve.Batcher((8, 32), 60000), reqs)
        assert all(r.error is None for r in mixed)
        mixed_pairs = {r.rid: r.pairs for r in mixed}
        alone_pairs = {}
        for r in reqs:
            solo = serve.Request(r.rid, r.sets, 0.0)
            out = serve.serve(ex, serve.Batcher((8, 32), 60000), [solo])
            alone_pairs[r.rid] = out[0].pairs
    finally:
        ex.close()
    assert mixed_pairs == alone_pairs
    # and the pairs are the oracle's
    lo = oc.layout(D, k, kg, *ab)
    perm = oc.permutation(D, 1)
    c_rows = oc.sketch(w["ids"], w["off"], lo, perm=perm)
    z = np.diff(lo[::kg]).astype(np.uint64)
    n_pairs = 0
    for r in reqs:
        ids, off = synth.pack_sets(r.sets)
        want = oc.query("hoph", oc.sketch(ids, off, lo, perm=perm), c_rows, kg, 7, 10, 1e-4, z=z)
        assert mixed_pairs[r.rid] == [tuple(int(v) for v in a) for a in want["accepted"]]
        n_pairs += want["count"]
    assert n_pairs > 0
