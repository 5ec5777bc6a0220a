"""GPU comparison (hoph_query_batch, hoph_pair_counts) against the CPU
oracle: accepted pairs, groups compared, matched bins and per-group
decision counts must be identical."""
import numpy as np
import pytest

from gpu_helpers import (device, oracle_rows, oracle_tuples, oracle_z, pairs_tuples,
                         planes_to_rows, rows_to_planes, to_dev, torch)  # noqa: F401
from oracle import oracle_c as oc
from paper_1805_11254_gb300 import hoph, shard, synth

pytestmark = pytest.mark.gpu

T = (7, 10)
EPS = 1e-4


@pytest.fixture(scope="module")
def small():
    return synth.small_parity_workload()


def _sketch_both(plan, w, dev):
    c = plan.sketch(to_dev(w["ids"], dev), to_dev(w["off"], dev), len(w["off"]) - 1)
    q = plan.sketch(to_dev(w["q_ids"], dev), to_dev(w["q_off"], dev), len(w["q_off"]) - 1)
    plan.check()
    return q, c


def _oracle_query(mode, q_rows, c_rows, kg, z, eps=EPS, rule="both", thr=T):
    return oc.query(mode, q_rows, c_rows, kg, thr[0], thr[1], eps, rule=rule,
                    z=np.asarray(z, dtype=np.uint64))


def _small_oracle(w, k, kg, ab, q=None, c=None):
    """The oracle's sketches of the small workload's queries and rows (psi
    from seed 1) and its group sizes; GPU planes q, c, when given, must
    equal them bit for bit."""
    D = w["D"]
    q_rows = oracle_rows(w["q_ids"], w["q_off"], D, k, kg, ab, 1)
    c_rows = oracle_rows(w["ids"], w["off"], D, k, kg, ab, 1)
    if q is not None:
        assert np.array_equal(planes_to_rows(q), q_rows)
    if c is not None:
        assert np.array_equal(planes_to_rows(c), c_rows)
    return q_rows, c_rows, oracle_z(D, k, kg, ab)


def _compare(plan, mode, q, c, nq, nr, want, strategy, G):
    """Run one strategy and compare with the oracle.  The value join is only
    offered when a pair without any match is rejected for every possible
    denominator; otherwise forcing it must fail with UNSUPPORTED."""
    plan.set_exec(strategy=strategy)
    try:
        pairs, n, st = plan.query(mode, q, nq, c, nr, capacity=1 << 16, stats=True)
    except hoph.HophError as e:
        assert strategy == 1 and e.code == hoph.HOPH_ERR_UNSUPPORTED
        return None
    assert n == want["count"]
    assert pairs_tuples(pairs) == oracle_tuples(want)
    hist = want["hist"]  # [groups compared][decision]
    for g in range(G):
        assert st.accepted[g] == hist[g + 1][1], ("accepted", g)
        assert st.rejected[g] == hist[g + 1][2], ("rejected", g)
    assert st.entering[0] == nq * nr
    return st


@pytest.mark.parametrize("strategy", [0, 1, -1])
@pytest.mark.parametrize("mode,ab,kg", [("goph", (0, 0), 32), ("hoph", (1, 1), 32),
                                        ("oph_full", (0, 0), 32), ("hoph", (1, 2), 32)])
def test_small_workload_parity(small, mode, ab, kg, strategy):
    """N = 5,000 sets over D = 2^16, k = 128, 50 planted queries, T = 0.7."""
    dev = device()
    D, k = small["D"], 128
    with hoph.Plan(D, k, kg, *ab, seed=1, thr=T, epsilon=EPS) as plan:
        q, c = _sketch_both(plan, small, dev)
        nq, nr = q.shape[1], c.shape[1]
        q_rows, c_rows, z = _small_oracle(small, k, kg, ab, q, c)
        want = _oracle_query(mode, q_rows, c_rows, kg, z)
        assert want["count"] > 0
        G = plan.G if mode in ("goph", "hoph") else 1
        _compare(plan, mode, q, c, nq, nr, want, strategy, G)


def test_minwise_query_parity(small):
    dev = device()
    D, mk = small["D"], 128
    with hoph.Plan(D, 128, 32, minwise_k=mk, seed=1, thr=T) as plan:
        c = plan.minwise(to_dev(small["ids"], dev), to_dev(small["off"], dev),
                         len(small["off"]) - 1)
        q = plan.minwise(to_dev(small["q_ids"], dev), to_dev(small["q_off"], dev),
                         len(small["q_off"]) - 1)
        plan.check()
        want = oc.query("minwise_full", q.cpu().numpy().view(np.uint32),
                        c.cpu().numpy().view(np.uint32), mk, T[0], T[1], EPS)
        pairs, n, _ = plan.query("minwise_full", q, q.shape[0], c, c.shape[0])
        assert n == want["count"] > 0
        assert pairs_tuples(pairs) == oracle_tuples(want)


def _mixed_sets(rng, n, D, empty_every=7):
    """Sets with many empty bins: tiny sets, empty sets, near duplicates."""
    base = []
    for i in range(n):
        s = 0 if i % empty_every == 0 else int(rng.integers(1, 40))
        base.append(rng.choice(D, s, replace=False).astype(np.uint32))
    out = list(base)
    for b in base[: n // 2]:
        if len(b) > 2:
            keep = b[: max(1, len(b) * 4 // 5)]
            out.append(np.concatenate([keep, rng.choice(D, 2).astype(np.uint32)]))
    return out


@pytest.mark.parametrize("rule", ["both", "either", "none"])
@pytest.mark.parametrize("eps", [0.0, 1e-3, 1.0])
@pytest.mark.parametrize("mode,ab", [("goph", (0, 0)), ("hoph", (1, 1)), ("oph_full", (0, 0))])
def test_rules_eps_and_empty_bins(mode, ab, rule, eps):
    dev = device()
    rng = np.random.default_rng(hash((mode, rule, eps)) & 0xFFFF)
    D, k, kg = 4096, 64, 16
    sets = _mixed_sets(rng, 120, D)
    ids, off = synth.pack_sets(sets)
    thr = (3, 5)
    with hoph.Plan(D, k, kg, *ab, seed=9, thr=thr, epsilon=eps, empty_rule=rule) as plan:
        d_ids, d_off = to_dev(ids, dev), to_dev(off, dev)
        c = plan.sketch(d_ids, d_off, len(sets))
        plan.check()
        rows = oracle_rows(ids, off, D, k, kg, ab, 9)
        assert np.array_equal(planes_to_rows(c), rows)
        z = oracle_z(D, k, kg, ab)
        want = _oracle_query(mode, rows, rows, kg, z, eps=eps, rule=rule, thr=thr)
        G = plan.G if mode != "oph_full" else 1
        for strategy in (0, -1, 1):
            _compare(plan, mode, c, c, len(sets), len(sets), want, strategy, G)


@pytest.mark.parametrize("n_rows", [1, 2, 31, 33, 257, 1001])
@pytest.mark.parametrize("n_q", [1, 3, 40])
def test_ragged_tiles_and_batch_sizes(small, n_rows, n_q):
    dev = device()
    D, k, kg = small["D"], 128, 32
    with hoph.Plan(D, k, kg, 1, 1, seed=1, thr=T) as plan:
        q_all, rows, z = _small_oracle(small, k, kg, (1, 1))
        # planted rows first so there are accepted pairs in range
        src = small["src"][:n_q]
        sel = np.concatenate([src, np.arange(n_rows)])[:n_rows]
        c_rows = rows[sel]
        q_rows = q_all[:n_q]
        want = _oracle_query("hoph", q_rows, c_rows, kg, z)
        for strategy in (0, 1):
            _compare(plan, "hoph", rows_to_planes(q_rows, kg, dev), rows_to_planes(c_rows, kg, dev),
                     n_q, n_rows, want, strategy, plan.G)


def test_empty_inputs_and_capacity_overflow(small):
    dev = device()
    D, k, kg = small["D"], 128, 32
    with hoph.Plan(D, k, kg, seed=1, thr=(1, 100), epsilon=EPS) as plan:
        q, c = _sketch_both(plan, small, dev)
        pairs, n, _ = plan.query("goph", q, 0, c, c.shape[1])
        assert n == 0
        pairs, n, _ = plan.query("goph", q, q.shape[1], c, 0)
        assert n == 0
        # T = 0.01 accepts nearly everything: more pairs than the buffer holds
        out = torch.empty((4, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        q_all, c_all, _ = _small_oracle(small, k, kg, (0, 0))
        rows, qrows = c_all[:100], q_all[:10]
        hoph.hoph_query_batch(plan.handle, "goph", rows_to_planes(qrows, kg, dev), 10,
                              rows_to_planes(rows, kg, dev), 100, out, 4, cnt)
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_ERR_CAPACITY
        want = oc.query("goph", qrows, rows, kg, 1, 100, EPS)
        assert int(cnt.item()) == want["count"] > 4
        got = set(pairs_tuples(out.cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)))
        assert got <= set(oracle_tuples(want))  # the 4 kept pairs are genuine


def test_goph_example_1_sketches_on_gpu():
    """Sec. 3.3 Example 1 (k'=100, n=10, T=0.6, eps=1e-4): matches 65, 5, 10,
    10 reject the pair after the fourth group; an identical pair is accepted
    when the remaining requirement falls into the lower tail."""
    from fractions import Fraction
    from oracle import hoph_ref as hr
    dev = device()
    kg, n = 100, 10
    s = np.zeros((1, kg * n), dtype=np.uint32)
    t = np.ones((2, kg * n), dtype=np.uint32)
    for g, m in enumerate([65, 5, 10, 10]):
        t[0, g * kg:g * kg + m] = 0
    t[1, :] = 0
    want0 = hr.goph_compare(s[0].tolist(), t[0].tolist(), kg, Fraction(3, 5), 1e-4)
    want1 = hr.goph_compare(s[0].tolist(), t[1].tolist(), kg, Fraction(3, 5), 1e-4)
    assert want0 == (hr.REJECT, 4, 90)
    assert want1[0] == hr.ACCEPT
    with hoph.Plan(100000, kg * n, kg, seed=1, thr=(3, 5), epsilon=1e-4) as plan:
        for strategy in (0, -1):
            plan.set_exec(strategy=strategy)
            pairs, cnt, st = plan.query("goph", rows_to_planes(s, kg, dev), 1,
                                        rows_to_planes(t, kg, dev), 2, stats=True)
            assert pairs_tuples(pairs) == [(0, 1, want1[1], want1[2])]
            assert st.rejected[3] == 1 and st.entering[3] == 2


def test_pair_counts_parity(small):
    dev = device()
    D, k, kg = small["D"], 128, 32
    with hoph.Plan(D, k, kg, 1, 1, seed=1) as plan:
        nr = 700
        qr, c_all, _ = _small_oracle(small, k, kg, (1, 1))
        cr = c_all[:nr]
        out = torch.empty((qr.shape[0], nr, plan.G, 3), dtype=torch.int16, device=dev)
        hoph.hoph_pair_counts(plan.handle, rows_to_planes(qr, kg, dev), qr.shape[0],
                              rows_to_planes(cr, kg, dev), nr, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint16)
        assert np.array_equal(got, oc.pair_counts(qr, cr, kg))


def test_identical_sets_always_accepted(small):
    dev = device()
    D, k, kg = small["D"], 128, 32
    with hoph.Plan(D, k, kg, 1, 1, seed=1, thr=(1, 1), epsilon=EPS) as plan:
        q, c = _sketch_both(plan, small, dev)
        rows = planes_to_rows(c)[:300]
        d = rows_to_planes(rows, kg, dev)
        pairs, n, _ = plan.query("hoph", d, 300, d, 300)
        got = {(int(p["query"]), int(p["row"])) for p in pairs}
        assert {(i, i) for i in range(300)} <= got


@pytest.mark.parametrize("kg,lpr,warps,stages", [(32, 1, 8, 2), (32, 2, 16, 2), (32, 1, 16, 3),
                                                 (32, 2, 3, 5), (64, 2, 16, 2), (64, 4, 16, 4),
                                                 (64, 2, 5, 3), (64, 4, 31, 2), (64, 4, 20, 2)])
def test_join_execution_knobs_do_not_change_results(small, kg, lpr, warps, stages):
    """Lanes per row, consumer warps and pipeline depth of the join filter
    are scheduling only: the accepted pairs stay the oracle's."""
    dev = device()
    D, k = small["D"], 128
    with hoph.Plan(D, k, kg, 1, 2, seed=1, thr=T, epsilon=EPS) as plan:
        q, c = _sketch_both(plan, small, dev)
        q_rows, c_rows, z = _small_oracle(small, k, kg, (1, 2), q, c)
        want = _oracle_query("hoph", q_rows, c_rows, kg, z)
        plan.set_exec(strategy=1, lanes_per_row=lpr, consumer_warps=warps, stages=stages)
        pairs, n, st = plan.query("hoph", q, q.shape[1], c, c.shape[1], stats=True)
        assert pairs_tuples(pairs) == oracle_tuples(want)
        assert st.strategy == 1 and st.rows_counted < c.shape[1]


def _planted_workload(n_rows, size_lo, size_hi, n_q, D, seed):
    sizes = synth.uniform_sizes(n_rows, size_lo, size_hi, seed)
    ids, off = synth.distinct_uniform_sets(sizes, D, seed + 1)
    rng = np.random.default_rng(seed + 2)
    src = rng.integers(0, n_rows, n_q // 2)
    planted, _ = synth.plant_near_duplicates([ids[off[r]:off[r + 1]] for r in src], D, 0.5,
                                             0.98, seed + 3)
    fresh_ids, fresh_off = synth.distinct_uniform_sets(
        synth.uniform_sizes(n_q - len(planted), size_lo, size_hi, seed + 4), D, seed + 5)
    qsets = planted + [fresh_ids[fresh_off[i]:fresh_off[i + 1]] for i in range(len(fresh_off) - 1)]
    q_ids, q_off = synth.pack_sets(qsets)
    return ids, off, q_ids, q_off


@pytest.mark.parametrize("case", ["hash61_2to1_k512", "oph_full_D2^22"])
def test_large_key_spaces_use_the_hashed_join(case):
    """Key spaces too large to index directly: a hashed group map (false hits
    only loosen the row filter) and, beyond 2^23 keys, an open-addressing key
    table.  Results stay the oracle's; the join must be the strategy used."""
    dev = device()
    if case.startswith("hash61"):
        D, k, kg, ab, mode = 1 << 32, 512, 128, (2, 1), "hoph"
        ids, off, q_ids, q_off = _planted_workload(1500, 1000, 3000, 64, D, 41)
        kw = dict(perm_kind=hoph.HOPH_PERM_HASH61)
    else:
        D, k, kg, ab, mode = 1 << 22, 128, 32, (0, 0), "oph_full"
        ids, off, q_ids, q_off = _planted_workload(3000, 100, 600, 48, D, 43)
        kw = {}
    thr = (7, 10)
    with hoph.Plan(D, k, kg, *ab, seed=7, thr=thr, epsilon=1e-4, **kw) as plan:
        c = plan.sketch(to_dev(ids, dev), to_dev(off, dev), len(off) - 1)
        q = plan.sketch(to_dev(q_ids, dev), to_dev(q_off, dev), len(q_off) - 1)
        plan.check()
        hashed = case.startswith("hash61")
        want_c = oracle_rows(ids, off, D, k, kg, ab, 7, hashed=hashed)
        want_q = oracle_rows(q_ids, q_off, D, k, kg, ab, 7, hashed=hashed)
        assert np.array_equal(planes_to_rows(c), want_c)
        assert np.array_equal(planes_to_rows(q), want_q)
        z = oracle_z(D, k, kg, ab)
        want = oc.query(mode, want_q, want_c, kg, thr[0], thr[1], 1e-4, z=z)
        assert want["count"] > 0
        plan.set_exec(strategy=1)
        pairs, n, st = plan.query(mode, q, q.shape[1], c, c.shape[1], stats=True)
        assert st.strategy == 1
        assert pairs_tuples(pairs) == oracle_tuples(want)


@pytest.mark.parametrize("world", [2, 3])
def test_row_shards_merge_to_the_whole_collection(small, world):
    """Each shard of rows queried alone (as a rank would), rows made global
    and merged, equals one query of the whole collection."""
    from paper_1805_11254_gb300 import shard
    dev = device()
    with hoph.Plan(small["D"], 128, 32, 1, 1, seed=1, thr=T, epsilon=EPS) as plan:
        q, c = _sketch_both(plan, small, dev)
        nq, n = q.shape[1], c.shape[1]
        whole, _, _ = plan.query(hoph.HOPH_MODE_HOPH, q, nq, c, n)
        parts = []
        for r in range(world):
            r0, r1 = shard.row_range(n, r, world)
            local = c[:, r0:r1, :].contiguous()
            run = shard.gpu_local_query(plan, hoph.HOPH_MODE_HOPH, q, nq, local, capacity=4)
            parts.append(shard.globalize(run(r0, r1), r0))
        assert len(whole) > 0
        assert np.array_equal(shard.merge_pairs(parts), whole)


@pytest.mark.parametrize("strategy", [0, 1, -1])
@pytest.mark.parametrize("ab", [(1, 1), (1, 2), (2, 1)])
def test_literal_weighting_parity(small, ab, strategy):
    """Algorithm 2's printed recursion (HOPH_WEIGHT_LITERAL) against the
    oracle's reduced-fraction route; for 1:1 it coincides with the space
    weighting at l = 1, for 1:2 it rejects near duplicates after group 1."""
    dev = device()
    D, k, kg = small["D"], 128, 32
    with hoph.Plan(D, k, kg, *ab, seed=1, thr=T, epsilon=EPS,
                   weighting=hoph.HOPH_WEIGHT_LITERAL) as plan:
        q, c = _sketch_both(plan, small, dev)
        nq, nr = q.shape[1], c.shape[1]
        q_rows, c_rows, z = _small_oracle(small, k, kg, ab, q, c)
        want = oc.query("hoph", q_rows, c_rows, kg, T[0], T[1], EPS, z=z, weighting="literal",
                        ab=ab)
        _compare(plan, "hoph", q, c, nq, nr, want, strategy, plan.G)



@pytest.mark.parametrize("strategy", [0, 1, -1])
@pytest.mark.parametrize("mode,ab,kg", [("goph", (0, 0), 32), ("hoph", (1, 2), 64),
                                        ("oph_full", (0, 0), 64), ("hoph", (1, 1), 32)])
def test_compact_planes_give_the_same_pairs(small, mode, ab, kg, strategy):
    """hoph_query_batch16 over uint16 planes: the oracle's pairs and
    per-group decision counts, through the dense scan and the value join
    (the join needs k' % 64 == 0 here; otherwise forcing it is UNSUPPORTED)."""
    dev = device()
    D, k = small["D"], 128
    with hoph.Plan(D, k, kg, *ab, seed=1, thr=T, epsilon=EPS) as plan:
        q, c = _sketch_both(plan, small, dev)
        q_rows, c_rows, z = _small_oracle(small, k, kg, ab, q, c)
        want = _oracle_query(mode, q_rows, c_rows, kg, z)
        q16 = plan.sketch16(to_dev(small["q_ids"], dev), to_dev(small["q_off"], dev), q.shape[1])
        c16 = plan.sketch16(to_dev(small["ids"], dev), to_dev(small["off"], dev), c.shape[1])
        plan.check()
        G = plan.G if mode in ("goph", "hoph") else 1
        plan.set_exec(strategy=strategy)
        try:
            pairs, n, st = plan.query(mode, q16, q.shape[1], c16, c.shape[1], capacity=1 << 16,
                                      stats=True)
        except hoph.HophError as e:
            assert strategy == 1 and e.code == hoph.HOPH_ERR_UNSUPPORTED
            return
        assert n == want["count"]
        assert pairs_tuples(pairs) == oracle_tuples(want)
        hist = want["hist"]
        for g in range(G):
            assert st.accepted[g] == hist[g + 1][1] and st.rejected[g] == hist[g + 1][2]
        if strategy >= 0:
            assert st.strategy == strategy


@pytest.mark.parametrize("batch", [777, 4096])
@pytest.mark.parametrize("mode,ab,kg", [("hoph", (1, 2), 64), ("goph", (0, 0), 32),
                                        ("oph_full", (0, 0), 64)])
def test_self_join_is_the_upper_triangle_of_the_all_pairs_query(small, mode, ab, kg, batch):
    """hoph_self_join over the 5,000 sets plus the 50 planted near duplicates
    appended as rows: exactly the oracle's accepted pairs (i, j) with i < j
    of the all-pairs comparison, in (i, j) order; ragged last block.  The
    statistics cover exactly the n (n - 1) / 2 pairs i < j, each decided in
    the group where the oracle decides it."""
    dev = device()
    D, k = small["D"], 128
    ids = np.concatenate([small["ids"], small["q_ids"]])
    off = np.concatenate([small["off"], small["off"][-1] + small["q_off"][1:]])
    n = len(off) - 1
    with hoph.Plan(D, k, kg, *ab, seed=1, thr=T, epsilon=EPS) as plan:
        c = plan.sketch(to_dev(ids, dev), to_dev(off, dev), n)
        plan.check()
        rows = oracle_rows(ids, off, D, k, kg, ab, 1)
        assert np.array_equal(planes_to_rows(c), rows)
        full = oc.query(mode, rows, rows, kg, T[0], T[1], EPS, z=oracle_z(D, k, kg, ab),
                        per_pair=True)
        want = full["accepted"]
        want = want[want[:, 0] < want[:, 1]]
        iu = np.triu_indices(n, 1)
        dec, grp = full["dec"][iu], full["groups"][iu]
        del full
        cap = 1 << 14
        out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(hoph.STATS_WORDS, dtype=torch.int64, device=dev)
        hoph.hoph_self_join(plan.handle, mode, c, n, batch, out, cap, cnt, st)
        plan.check()
        m = int(cnt.item())
        got = out[:m].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
        stats = hoph.hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes())
        G = plan.G if mode != "oph_full" else 1
    assert len(want) > 5  # the planted pairs at J >= T
    assert m == len(want)
    assert [(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"])) for p in got] \
        == [tuple(int(x) for x in w) for w in want]
    assert stats.entering[0] == n * (n - 1) // 2
    for g in range(G):
        assert stats.accepted[g] == np.count_nonzero((grp == g + 1) & (dec == 1)), ("acc", g)
        assert stats.rejected[g] == np.count_nonzero((grp == g + 1) & (dec == 2)), ("rej", g)


@pytest.fixture(scope="module")
def self_join_case(small):
    """(1:2)HOPH, k' = 64 over the 5,000 sets plus the 50 planted near
    duplicates: the collection and the oracle's accepted upper-triangle pairs
    with per-group decision counts."""
    D, k, kg, ab = small["D"], 128, 64, (1, 2)
    ids = np.concatenate([small["ids"], small["q_ids"]])
    off = np.concatenate([small["off"], small["off"][-1] + small["q_off"][1:]])
    n = len(off) - 1
    lo = oc.layout(D, k, kg, *ab)
    rows = oc.sketch(ids, off, lo, perm=oc.permutation(D, 1))
    z = np.diff(lo[::kg]).astype(np.uint64)
    full = oc.query("hoph", rows, rows, kg, T[0], T[1], EPS, z=z, per_pair=True)
    want = full["accepted"]
    want = [tuple(int(x) for x in w) for w in want[want[:, 0] < want[:, 1]]]
    iu = np.triu_indices(n, 1)
    dec, grp = full["dec"][iu], full["groups"][iu]
    acc = [int(np.count_nonzero((grp == g + 1) & (dec == 1))) for g in range(k // kg)]
    rej = [int(np.count_nonzero((grp == g + 1) & (dec == 2))) for g in range(k // kg)]
    return dict(D=D, k=k, kg=kg, ab=ab, ids=ids, off=off, n=n, want=want, acc=acc, rej=rej)


def _run_self_join(plan, c, n, batch, cap, dev, stream=None):
    out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    st = torch.zeros(hoph.STATS_WORDS, dtype=torch.int64, device=dev)
    hoph.hoph_self_join(plan.handle, hoph.HOPH_MODE_HOPH, c, n, batch, out, cap, cnt, st, stream)
    return out, cnt, st


def _self_join_result(out, cnt, st):
    m = int(cnt.item())
    got = out[:m].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
    stats = hoph.hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes())
    return ([(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"])) for p in got],
            stats)


@pytest.mark.parametrize("lanes", [1, 3, 4, 8])
def test_self_join_blocks_in_flight_keep_the_result(self_join_case, lanes):
    """join_lanes = 1, 3, 4 (blocks of 300 rows on that many of the plan's
    streams at once), through Plan.self_join: the oracle's upper-triangle
    pairs, in order, and its per-group decision counts."""
    dev = device()
    w = self_join_case
    with hoph.Plan(w["D"], w["k"], w["kg"], *w["ab"], seed=1, thr=T, epsilon=EPS) as plan:
        c = plan.sketch(to_dev(w["ids"], dev), to_dev(w["off"], dev), w["n"])
        plan.update_exec(join_lanes=lanes)
        pairs, m, stats = plan.self_join("hoph", c, w["n"], batch=300, stats=True)
        got = [(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"]))
               for p in pairs]
    assert m == len(got)
    assert got == w["want"]
    assert stats.entering[0] == w["n"] * (w["n"] - 1) // 2
    assert list(stats.accepted[:len(w["acc"])]) == w["acc"]
    assert list(stats.rejected[:len(w["rej"])]) == w["rej"]


@pytest.mark.parametrize("knobs", [dict(strategy=1, lanes_per_row=0),
                                   dict(strategy=1, lanes_per_row=32, consumer_warps=5,
                                        tile_rows=96),
                                   dict(strategy=1, lanes_per_row=4),
                                   dict(strategy=0)])
def test_compact_self_join_gives_the_oracle_pairs(self_join_case, knobs):
    """hoph_self_join16 over compact 16-bit planes, blocks of 300 rows on
    three streams, through the striped filter (the library's choice and
    forced, ragged tiles), the lanes-over-rows filter and the dense scan: the
    oracle's upper-triangle pairs in order and its per-group decision
    counts, as for the uint32 planes."""
    dev = device()
    w = self_join_case
    with hoph.Plan(w["D"], w["k"], w["kg"], *w["ab"], seed=1, thr=T, epsilon=EPS) as plan:
        c16 = plan.sketch16(to_dev(w["ids"], dev), to_dev(w["off"], dev), w["n"])
        plan.set_exec(join_lanes=3, **knobs)
        pairs, m, stats = plan.self_join("hoph", c16, w["n"], batch=300, stats=True)
        plan.check()
        got = [(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"]))
               for p in pairs]
    assert c16.dtype == torch.int16
    assert m == len(got)
    assert got == w["want"]
    assert stats.entering[0] == w["n"] * (w["n"] - 1) // 2
    assert list(stats.accepted[:len(w["acc"])]) == w["acc"]
    assert list(stats.rejected[:len(w["rej"])]) == w["rej"]


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("parts", [2, 3, 24])
def test_self_join_parts_add_up_to_the_self_join(self_join_case, compact, parts):
    """hoph_self_join_part, blocks of 300 rows dealt to 2, 3 or 24 parts (as
    over that many GPUs, each holding the whole collection; with 24, parts
    beyond the 17 blocks get none): every part's pairs in (query, row) order,
    their union the oracle's upper-triangle pairs and their statistics
    summing to the oracle's decision counts."""
    dev = device()
    w = self_join_case
    with hoph.Plan(w["D"], w["k"], w["kg"], *w["ab"], seed=1, thr=T, epsilon=EPS) as plan:
        sk = plan.sketch16 if compact else plan.sketch
        c = sk(to_dev(w["ids"], dev), to_dev(w["off"], dev), w["n"])
        plan.update_exec(join_lanes=2)
        chunks, acc, rej, entering = [], None, None, 0
        for part in range(parts):
            pairs, m, st = plan.self_join("hoph", c, w["n"], batch=300, stats=True, part=part,
                                          parts=parts)
            got = [(int(p["query"]), int(p["row"])) for p in pairs]
            assert m == len(got) and got == sorted(got)
            assert all(q // 300 in shard.self_join_blocks(w["n"], 300, part, parts)
                       for q, _ in got)
            chunks.append(pairs)
            a, r = np.asarray(st.accepted, dtype=np.int64), np.asarray(st.rejected, dtype=np.int64)
            acc = a if acc is None else acc + a
            rej = r if rej is None else rej + r
            entering += st.entering[0]
        plan.check()
    merged = shard.merge_pairs(chunks)
    assert [(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"]))
            for p in merged] == w["want"]
    assert entering == w["n"] * (w["n"] - 1) // 2
    assert list(acc[:len(w["acc"])]) == w["acc"]
    assert list(rej[:len(w["rej"])]) == w["rej"]


def test_self_join_with_lanes_replays_from_a_graph(self_join_case):
    """The self-join's fork onto the plan's streams and join back, captured
    in a CUDA graph (after one eager call has created the streams) and
    replayed twice: the oracle's pairs each time."""
    dev = device()
    w = self_join_case
    with hoph.Plan(w["D"], w["k"], w["kg"], *w["ab"], seed=1, thr=T, epsilon=EPS) as plan:
        c = plan.sketch(to_dev(w["ids"], dev), to_dev(w["off"], dev), w["n"])
        plan.update_exec(join_lanes=2)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            bufs = _run_self_join(plan, c, w["n"], 400, 1 << 14, dev, side)
            side.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                hoph.hoph_self_join(plan.handle, hoph.HOPH_MODE_HOPH, c, w["n"], 400, bufs[0],
                                    1 << 14, bufs[1], None, side)
        torch.cuda.synchronize()
        for _ in range(2):
            bufs[0].zero_()
            g.replay()
            torch.cuda.synchronize()
            got, _ = _self_join_result(*bufs)
            assert got == w["want"]
        plan.check()


def test_self_join_edges_capacity_and_arguments(self_join_case):
    """Fewer than two rows: no pairs.  An output buffer of 3 pairs: the
    device reports HOPH_ERR_CAPACITY, the count is the oracle's full count,
    and the 3 kept pairs are genuine (sorted among themselves).  Bad batch
    sizes and MinWise are refused on the host before anything runs."""
    dev = device()
    w = self_join_case
    with hoph.Plan(w["D"], w["k"], w["kg"], *w["ab"], seed=1, thr=T, epsilon=EPS) as plan:
        c = plan.sketch(to_dev(w["ids"], dev), to_dev(w["off"], dev), w["n"])
        plan.check()
        for n in (0, 1):
            out, cnt, _ = _run_self_join(plan, c, n, 64, 4, dev)
            plan.check()
            assert int(cnt.item()) == 0
        out, cnt, _ = _run_self_join(plan, c, w["n"], 500, 3, dev)
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_ERR_CAPACITY
        assert int(cnt.item()) == len(w["want"])
        kept = [(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"]))
                for p in out.cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)]
        assert kept == sorted(kept) and set(kept) <= set(w["want"])
        out = torch.empty((4, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        for batch in (0, 4097):
            with pytest.raises(hoph.HophError) as e:
                hoph.hoph_self_join(plan.handle, hoph.HOPH_MODE_HOPH, c, w["n"], batch, out, 4,
                                    cnt)
            assert e.value.code == hoph.HOPH_ERR_PARAM
        with pytest.raises(hoph.HophError) as e:
            hoph.hoph_self_join(plan.handle, "minwise_full", c, w["n"], 64, out, 4, cnt)
        assert e.value.code == hoph.HOPH_ERR_UNSUPPORTED
        plan.check()


def test_compact_planes_with_a_hashed_join():
    """Compact planes over a key space that needs the hashed group map and
    the key table (D = 256 x 65,535, k = 256 bins of 65,535 values, the
    widest a 16-bit offset allows; all four groups of 64 bins scanned as
    plain OPH): the oracle's pairs through the join."""
    dev = device()
    D, k, kg = 256 * 65535, 256, 64
    ids, off, q_ids, q_off = _planted_workload(2000, 200, 900, 40, D, 47)
    thr = (7, 10)
    with hoph.Plan(D, k, kg, seed=9, thr=thr, epsilon=1e-4) as plan:
        assert plan.info.max_bin_width == 0xFFFF
        c = plan.sketch(to_dev(ids, dev), to_dev(off, dev), len(off) - 1)
        q = plan.sketch(to_dev(q_ids, dev), to_dev(q_off, dev), len(q_off) - 1)
        c16 = plan.sketch16(to_dev(ids, dev), to_dev(off, dev), len(off) - 1)
        q16 = plan.sketch16(to_dev(q_ids, dev), to_dev(q_off, dev), len(q_off) - 1)
        plan.check()
        want_q = oracle_rows(q_ids, q_off, D, k, kg, (0, 0), 9)
        want_c = oracle_rows(ids, off, D, k, kg, (0, 0), 9)
        assert np.array_equal(planes_to_rows(q), want_q)
        assert np.array_equal(planes_to_rows(c), want_c)
        want = oc.query("oph_full", want_q, want_c, kg, thr[0], thr[1], 1e-4,
                        z=oracle_z(D, k, kg))
        assert want["count"] > 0
        plan.set_exec(strategy=1)
        pairs, n, st = plan.query("oph_full", q16, q16.shape[1], c16, c16.shape[1], stats=True)
        assert st.strategy == 1
        assert pairs_tuples(pairs) == oracle_tuples(want)


def test_autotuner_keeps_the_result_and_sets_the_fastest_knobs(small):
    """autotune.tune_query over the join and dense settings: every setting
    it times returns the oracle's pairs (it raises otherwise), the chosen one
    is left on the plan, and the pairs after tuning are still the oracle's;
    tune_sketch likewise for the sketch's CTA-size knob."""
    from paper_1805_11254_gb300 import autotune
    dev = device()
    D, k, kg, ab = small["D"], 128, 32, (1, 1)
    with hoph.Plan(D, k, kg, *ab, seed=1, thr=T, epsilon=EPS) as plan:
        q, c = _sketch_both(plan, small, dev)
        nq, nr = q.shape[1], c.shape[1]
        cap = 1 << 14
        out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        best, times = autotune.tune_query(plan, "hoph", q, nq, c, nr, out, cap, cnt,
                                          finalists=2, rounds=2)
        assert best is not None and len(times) >= 2
        assert all(plan.exec_kwargs[kk] == v for kk, v in best.items())
        pairs, n, _ = plan.query("hoph", q, nq, c, nr)
        q_rows, c_rows, z = _small_oracle(small, k, kg, ab, q, c)
        want = _oracle_query("hoph", q_rows, c_rows, kg, z)
        assert pairs_tuples(pairs) == oracle_tuples(want)
        d_ids, d_off = to_dev(small["ids"], dev), to_dev(small["off"], dev)
        sk = torch.empty_like(c)
        bits, btimes = autotune.tune_sketch(plan, d_ids, d_off, nr, sk, finalists=2, rounds=2)
        assert plan.exec_kwargs["sketch_cta_bits"] == bits and len(btimes) >= 2
        assert torch.equal(sk, c)


@pytest.mark.parametrize("knobs", [dict(consumer_warps=16, stages=2, tile_rows=256),
                                   dict(consumer_warps=16, stages=4, tile_rows=64),
                                   dict(consumer_warps=5, stages=3, tile_rows=96)])
@pytest.mark.parametrize("k,kg,compact", [(128, 32, False), (256, 64, False), (256, 128, False),
                                          (256, 64, True), (256, 128, True)])
def test_striped_filter_keeps_the_oracle_pairs(small, k, kg, compact, knobs):
    """The join filter over the bank-striped group map (lanes_per_row = 32:
    a warp per row, lane l reading words l, l + 32, ...), for 32, 64 and 128
    scanned bins, uint32 and compact planes, ragged last tiles: the oracle's
    pairs and per-group decision counts; with too few row bytes for whole
    lanes (32 compact bins) it is refused."""
    dev = device()
    D, ab = small["D"], (1, 2)
    with hoph.Plan(D, k, kg, *ab, seed=1, thr=T, epsilon=EPS) as plan:
        q_rows, c_rows, z = _small_oracle(small, k, kg, ab)
        want = _oracle_query("hoph", q_rows, c_rows, kg, z)
        assert want["count"] > 0
        if compact:
            q = plan.sketch16(to_dev(small["q_ids"], dev), to_dev(small["q_off"], dev),
                              len(q_rows))
            c = plan.sketch16(to_dev(small["ids"], dev), to_dev(small["off"], dev), len(c_rows))
        else:
            q, c = _sketch_both(plan, small, dev)
        plan.check()
        plan.set_exec(strategy=1, lanes_per_row=32, **knobs)
        pairs, n, st = plan.query("hoph", q, q.shape[1], c, c.shape[1], capacity=1 << 16,
                                  stats=True)
        assert st.strategy == 1
        assert n == want["count"]
        assert pairs_tuples(pairs) == oracle_tuples(want)
        for g in range(plan.G):
            assert st.accepted[g] == want["hist"][g + 1][1]
            assert st.rejected[g] == want["hist"][g + 1][2]
    with hoph.Plan(D, 128, 32, *ab, seed=1, thr=T, epsilon=EPS) as plan:
        q16 = plan.sketch16(to_dev(small["q_ids"], dev), to_dev(small["q_off"], dev), 50)
        c16 = plan.sketch16(to_dev(small["ids"], dev), to_dev(small["off"], dev), 5000)
        plan.set_exec(strategy=1, lanes_per_row=32)
        with pytest.raises(hoph.HophError) as e:
            plan.query("hoph", q16, 50, c16, 5000)
        assert e.value.code == hoph.HOPH_ERR_UNSUPPORTED


@pytest.mark.parametrize("lanes_per_row", [0, 32])
def test_value_join_when_rows_hit_most_queries(lanes_per_row):
    """Sketches over two values per bin, so every row hits nearly all of 600
    queries in most bins: the value join passes most rows, and its candidate
    counting walks long query lists for each of them and drains its
    survivor list many times; (1:2)HOPH at T = 7/10 rejects pairs after the
    first group and takes others on.  The oracle's pairs and per-group
    decision counts."""
    dev = device()
    rng = np.random.default_rng(78)
    D, k, kg, ab, nq, nr = 1 << 16, 256, 64, (1, 2), 600, 1500
    q_rows = rng.integers(0, 2, (nq, k)).astype(np.uint32)
    c_rows = rng.integers(0, 2, (nr, k)).astype(np.uint32)
    c_rows[:40] = q_rows[:40]  # some exact duplicates
    c_rows[rng.random((nr, k)) < 0.05] = hoph.HOPH_EMPTY_VALUE
    want = oc.query("hoph", q_rows, c_rows, kg, T[0], T[1], EPS, z=oracle_z(D, k, kg, ab))
    assert want["count"] >= 40
    with hoph.Plan(D, k, kg, *ab, seed=1, thr=T, epsilon=EPS) as plan:
        q, c = rows_to_planes(q_rows, kg, dev), rows_to_planes(c_rows, kg, dev)
        plan.set_exec(strategy=1, lanes_per_row=lanes_per_row)
        pairs, n, st = plan.query("hoph", q, nq, c, nr, capacity=1 << 16, stats=True)
        assert st.strategy == 1
        assert st.rows_counted > nr // 2
        assert n == want["count"]
        got = np.stack([pairs["query"].astype(np.int64), pairs["row"],
                        pairs["groups"].astype(np.int64), pairs["matches"].astype(np.int64)], 1)
        assert np.array_equal(got, want["accepted"])
        hist = want["hist"]
        for g in range(plan.G):
            assert st.accepted[g] == hist[g + 1][1] and st.rejected[g] == hist[g + 1][2]
    assert hist[1][2] > 0 and hist[2:].sum() > 0  # group 1 rejects some pairs, others go on


def test_over_a_million_accepted_pairs_come_out_in_order():
    """Over a million accepted pairs (sketches over two values per bin, so about
    half the bins of a pair match; T = 2/5): a capacity above the one-CTA
    sort's limit takes the many-CTA run sort and merge passes, and the output
    is exactly the oracle's accepted pairs in (query, row) order, with the
    groups compared and matched bins of each; a capacity one short reports
    HOPH_ERR_CAPACITY with the full count.  (Dense scan: at k' = 32 and
    T = 2/5 a pair without a match is not rejected at every denominator, so
    the value join is not offered.)"""
    dev = device()
    rng = np.random.default_rng(77)
    D, k, kg, nq, nr = 1 << 16, 64, 32, 1200, 1100
    q_rows = rng.integers(0, 2, (nq, k)).astype(np.uint32)
    c_rows = rng.integers(0, 2, (nr, k)).astype(np.uint32)
    q_rows[rng.random((nq, k)) < 0.05] = hoph.HOPH_EMPTY_VALUE
    c_rows[rng.random((nr, k)) < 0.05] = hoph.HOPH_EMPTY_VALUE
    thr = (2, 5)
    want = oc.query("goph", q_rows, c_rows, kg, thr[0], thr[1], EPS)
    assert want["count"] > 1_000_000
    with hoph.Plan(D, k, kg, seed=1, thr=thr, epsilon=EPS) as plan:
        q, c = rows_to_planes(q_rows, kg, dev), rows_to_planes(c_rows, kg, dev)
        pairs, n, st = plan.query("goph", q, nq, c, nr, capacity=want["count"] + 5, stats=True)
        assert n == want["count"]
        got = np.stack([pairs["query"].astype(np.int64), pairs["row"],
                        pairs["groups"].astype(np.int64), pairs["matches"].astype(np.int64)], 1)
        assert np.array_equal(got, want["accepted"])
        hist = want["hist"]
        for g in range(plan.G):
            assert st.accepted[g] == hist[g + 1][1] and st.rejected[g] == hist[g + 1][2]
        out = torch.empty((want["count"] - 1, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        hoph.hoph_query_batch(plan.handle, "goph", q, nq, c, nr, out, want["count"] - 1, cnt)
        assert hoph.hoph_sync_status(plan.handle) == hoph.HOPH_ERR_CAPACITY
        assert int(cnt.item()) == want["count"]
