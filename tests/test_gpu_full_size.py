"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times, on outputs the oracle can compute one by one:

* the batched (1:2)HOPH query of 1,024 query sets against 10^7 resident
  k = 256 sketches (value join, 16 consumer warps; and over compact 16-bit
  planes): sampled rows against every query;
* the shingle regime (D = 2^32, hashed psi, (2:1)HOPH, k = 512) against
  5*10^6 sketches generated inside the kernel;
* the 10^6-set sketch with Zipf IDs, with the default and the tuned
  size from which a set gets a whole CTA: sampled sets, all the largest ones;
* the self-join of 10^6 rows plus 1,000 planted near duplicates: every
  reported pair, every planted pair and a random sample of pairs.

The collection's IDs come from the counter generator on the device; the
oracle regenerates the sampled sets on the host (synth's twin of the
generator) and sketches and decides them itself.
"""
import numpy as np
import pytest

from gpu_helpers import device, planes_to_rows, to_dev, torch
from oracle import oracle_c as oc
from paper_1805_11254_gb300 import hoph, synth

pytestmark = pytest.mark.gpu

D = 1 << 20
K, KG, AB = 256, 64, (1, 2)
T = (7, 10)
EPS = 1e-4
PERM_SEED, COLL_SEED, Q_SEED, PLANT_SEED, SKETCH_SEED = 1, 11, 12, 13, 21


def _row_ids(coll_seed, off, r):
    return synth.counter_ids(coll_seed, int(off[r]), int(off[r + 1] - off[r]), D)


def _oracle_rows(coll_seed, off, rows, lo, perm):
    ids, offs = synth.pack_sets([_row_ids(coll_seed, off, int(r)) for r in rows])
    return oc.sketch(ids, offs, lo, perm)


def _device_rows(planes, rows, dev):
    idx = torch.from_numpy(np.asarray(rows, dtype=np.int64)).to(dev)
    return planes_to_rows(planes.index_select(1, idx))


def test_full_size_query_matches_the_oracle_on_sampled_rows():
    """1,024 query sets (10% planted at J 0.6-0.95) against 10^7 rows: the
    sketches of 4,096 random rows, of every row the GPU reported and of
    every planted source row equal the oracle's, the accepted pairs among
    those rows (each against all 1,024 queries) are exactly the oracle's,
    and the statistics count all 1.024 x 10^10 pairs.  The same over compact
    16-bit planes (the offsets in 16 bits, the same pairs)."""
    dev = device()
    n, nq = 10_000_000, 1024
    off = synth.offsets_from_sizes(synth.counter_collection_sizes(n, COLL_SEED))
    qw = synth.query_batch(nq, 0.1, D, COLL_SEED, off, 0.6, 0.95, Q_SEED, PLANT_SEED)
    lo = oc.layout(D, K, KG, *AB)
    perm = oc.permutation(D, PERM_SEED)
    with hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=T, epsilon=EPS) as plan:
        n_ids = int(off[-1])
        d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(COLL_SEED, 0, n_ids, D, 0, None, 0, d_ids)
        d_off = to_dev(off, dev)
        planes = plan.sketch(d_ids, d_off, n)
        planes16 = plan.sketch16(d_ids, d_off, n)
        del d_ids
        torch.cuda.empty_cache()
        d_qids, d_qoff = to_dev(qw["q_ids"], dev), to_dev(qw["q_off"], dev)
        q = plan.sketch(d_qids, d_qoff, nq)
        q16 = plan.sketch16(d_qids, d_qoff, nq)
        plan.check()
        plan.set_exec(strategy=1, lanes_per_row=0, consumer_warps=16, stages=3)
        pairs, m, st = plan.query(hoph.HOPH_MODE_HOPH, q, nq, planes, n, stats=True)
        # compact 16-bit planes, in both shapes the benchmark's tuner has picked
        # for them (16 warps, two lanes per row; 31 warps, four lanes per row)
        compact = []
        for lpr, cw, stg in ((0, 16, 3), (4, 31, 2)):
            plan.set_exec(strategy=1, lanes_per_row=lpr, consumer_warps=cw, stages=stg)
            compact.append(plan.query(hoph.HOPH_MODE_HOPH, q16, nq, planes16, n)[:2])
        G = plan.G
        rng = np.random.default_rng(5)
        src = qw["src"][qw["src"] >= 0]
        sample = np.unique(np.concatenate([rng.choice(n, 4096, replace=False),
                                           pairs["row"].astype(np.int64),
                                           *[p["row"].astype(np.int64) for p, _ in compact],
                                           src]))
        got_rows = _device_rows(planes, sample, dev)
        idx = torch.from_numpy(sample).to(dev)
        got_rows16 = planes16.index_select(1, idx).cpu().numpy().view(np.uint16) \
            .transpose(1, 0, 2).reshape(len(sample), -1)
        got_q = planes_to_rows(q)
        del planes, planes16
        torch.cuda.empty_cache()
    want_rows = _oracle_rows(COLL_SEED, off, sample, lo, perm)
    want_q = oc.sketch(qw["q_ids"], qw["q_off"], lo, perm)
    assert np.array_equal(got_q, want_q)
    assert np.array_equal(got_rows, want_rows)
    z = np.diff(lo[::KG]).astype(np.uint64)
    want = oc.query("hoph", want_q, want_rows, KG, T[0], T[1], EPS, z=z)["accepted"]
    want_set = {(int(a), int(sample[b]), int(g), int(mm)) for a, b, g, mm in want}
    got_set = {(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"]))
               for p in pairs}
    assert m == len(pairs) and m > 0
    assert got_set == want_set  # every reported row is in the sample
    # compact planes: the offsets in 16 bits (empty 0xFFFF), the same pairs
    want16 = np.where(want_rows == hoph.HOPH_EMPTY_VALUE, hoph.HOPH_EMPTY_VALUE16, want_rows)
    assert np.array_equal(got_rows16, want16.astype(np.uint16))
    for pairs16, m16 in compact:
        assert m16 == m and {(int(p["query"]), int(p["row"]), int(p["groups"]),
                              int(p["matches"])) for p in pairs16} == want_set
    assert sum(1 for p in want_set if p[1] in set(src.tolist())) > 0
    assert st.entering[0] == nq * n
    assert sum(st.accepted[g] for g in range(G)) == m
    assert sum(st.accepted[g] + st.rejected[g] for g in range(G)) == nq * n


@pytest.mark.parametrize("bits", [0, 13, 14])
def test_full_size_sketch_matches_the_oracle_on_sampled_sets(bits):
    """10^6 sets, lognormal sizes (median 300, sigma 1, [10, 20000]), Zipf(1.1)
    IDs over 2^20, k = 256: 2,000 random sets and the 256 largest (which a
    whole CTA sketches) equal the oracle's sketches, with the default and
    the tuned CTA-size knob."""
    dev = device()
    n = 1_000_000
    sizes = synth.lognormal_sizes(n, 300, 1.0, 10, 20000, SKETCH_SEED)
    off = synth.offsets_from_sizes(sizes)
    cdf = synth.zipf_cdf(D, 1.1)
    lo = oc.layout(D, K, K)
    perm = oc.permutation(D, PERM_SEED)
    with hoph.Plan(D, K, K, seed=PERM_SEED, thr=T, epsilon=EPS) as plan:
        n_ids = int(off[-1])
        d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(SKETCH_SEED, 0, n_ids, D, 1, torch.from_numpy(cdf).to(dev),
                            len(cdf), d_ids)
        plan.update_exec(sketch_cta_bits=bits)
        sk = plan.sketch(d_ids, to_dev(off, dev), n)
        plan.check()
        rng = np.random.default_rng(6)
        sample = np.unique(np.concatenate([rng.choice(n, 2000, replace=False),
                                           np.argsort(sizes, kind="stable")[-256:]]))
        got = _device_rows(sk, sample, dev)
    ids, offs = synth.pack_sets([synth.counter_zipf_ids(SKETCH_SEED, int(off[r]),
                                                        int(off[r + 1] - off[r]), cdf)
                                 for r in sample])
    assert np.array_equal(got, oc.sketch(ids, offs, lo, perm))


def test_full_size_self_join_on_reported_planted_and_random_pairs():
    """hoph_self_join over the first 10^6 rows of the query workload's
    collection plus 1,000 planted near duplicates (J 0.6-0.95) of random rows
    among them, blocks of 1,536 rows: every reported pair is one the oracle
    accepts, with its groups and matches; every planted pair the oracle
    accepts is reported; so is every accepted pair of 4,000 random pairs;
    and the statistics cover exactly the n (n - 1) / 2 pairs.  The compact
    self-join (hoph_self_join16, the striped filter) gives the same pairs and
    statistics."""
    dev = device()
    n_base, n_pl = 1_000_000, 1000
    off_all = synth.offsets_from_sizes(synth.counter_collection_sizes(10_000_000, COLL_SEED))
    off = off_all[:n_base + 1]
    rng = np.random.default_rng(PLANT_SEED + 7)
    src = np.sort(rng.choice(n_base, n_pl, replace=False))
    bases = [_row_ids(COLL_SEED, off, r) for r in src]
    planted, _ = synth.plant_near_duplicates(bases, D, 0.6, 0.95, PLANT_SEED + 8)
    p_ids, p_off = synth.pack_sets(planted)
    n = n_base + n_pl
    lo = oc.layout(D, K, KG, *AB)
    perm = oc.permutation(D, PERM_SEED)
    z = np.diff(lo[::KG]).astype(np.uint64)
    with hoph.Plan(D, K, KG, *AB, seed=PERM_SEED, thr=T, epsilon=EPS) as plan:
        n_ids = int(off[n_base])
        d_ids = torch.empty(n_ids, dtype=torch.int32, device=dev)
        hoph.hoph_synth_ids(COLL_SEED, 0, n_ids, D, 0, None, 0, d_ids)
        base = plan.sketch(d_ids, to_dev(off, dev), n_base)
        base16 = plan.sketch16(d_ids, to_dev(off, dev), n_base)
        del d_ids
        pl = plan.sketch(to_dev(p_ids, dev), to_dev(p_off, dev), n_pl)
        pl16 = plan.sketch16(to_dev(p_ids, dev), to_dev(p_off, dev), n_pl)
        planes = torch.cat([base, pl], dim=1).contiguous()
        planes16 = torch.cat([base16, pl16], dim=1).contiguous()
        del base, pl, base16, pl16
        plan.check()
        cap = 1 << 20
        out = torch.empty((cap, 2), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(hoph.STATS_WORDS, dtype=torch.int64, device=dev)
        hoph.hoph_self_join(plan.handle, hoph.HOPH_MODE_HOPH, planes, n, 1536, out, cap, cnt, st)
        plan.check()
        m = int(cnt.item())
        got = out[:m].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
        stats = hoph.hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes())
        G = plan.G
        del planes
        st.zero_()
        hoph.hoph_self_join16(plan.handle, hoph.HOPH_MODE_HOPH, planes16, n, 1536, out, cap, cnt,
                              st)
        plan.check()
        got16 = out[:int(cnt.item())].cpu().numpy().view(hoph.PAIR_DTYPE).reshape(-1)
        stats16 = hoph.hoph_stats.from_buffer_copy(st.cpu().numpy().tobytes())
        del planes16
        torch.cuda.empty_cache()
    assert np.array_equal(got16, got)
    for f in ("entering", "accepted", "rejected"):
        assert list(getattr(stats16, f)) == list(getattr(stats, f))

    def ids_of(r):
        return _row_ids(COLL_SEED, off, r) if r < n_base else planted[r - n_base]

    def decide(pairs_ij):
        """oracle (accepted, groups, matches) of each pair (i, j)."""
        rows = sorted({r for p in pairs_ij for r in p})
        pos = {r: i for i, r in enumerate(rows)}
        ids, offs = synth.pack_sets([ids_of(r) for r in rows])
        sk = oc.sketch(ids, offs, lo, perm)
        res = []
        for i, j in pairs_ij:
            w = oc.query("hoph", sk[pos[i]][None], sk[pos[j]][None], KG, T[0], T[1], EPS, z=z,
                         threads=1)
            a = w["accepted"]
            res.append((True, int(a[0][2]), int(a[0][3])) if len(a) else (False, 0, 0))
        return res

    assert m > n_pl // 2
    got_pairs = [(int(p["query"]), int(p["row"])) for p in got]
    assert all(i < j for i, j in got_pairs) and got_pairs == sorted(got_pairs)
    for p, (acc, g, mm) in zip(got, decide(got_pairs)):
        assert acc and (g, mm) == (int(p["groups"]), int(p["matches"]))
    reported = set(got_pairs)
    planted_pairs = [(int(src[i]), n_base + i) for i in range(n_pl)]
    for pr, (acc, _, _) in zip(planted_pairs, decide(planted_pairs)):
        assert acc == (pr in reported)
    rng = np.random.default_rng(8)
    a, b = rng.integers(0, n, 4000), rng.integers(0, n, 4000)
    rand = [(int(min(x, y)), int(max(x, y))) for x, y in zip(a, b) if x != y]
    for pr, (acc, _, _) in zip(rand, decide(rand)):
        assert acc == (pr in reported)
    assert stats.entering[0] == n * (n - 1) // 2
    assert sum(stats.accepted[g] for g in range(G)) == m


def test_full_size_shingle_regime_on_sampled_rows():
    """IDs uniform over 2^32, psi the 2-universal hash mod 2^61-1, (2:1)HOPH
    with k = 512, k' = 128: the 5*10^6-set collection (sizes U[1000,
    100000]) generated and sketched inside the kernel, and one batch of
    1,024 query sets (32 planted near duplicates at J 0.75-0.98) through the
    hashed join in the benchmark's tuned shape.  512 random rows, every
    reported row and every planted source row: sketches equal the oracle's
    and, against all 1,024 queries, so do the accepted pairs."""
    dev = device()
    D4, K4, KG4, AB4 = 1 << 32, 512, 128, (2, 1)
    seed_c, seed_q, n, nq, n_pl = 31, 32, 5_000_000, 1024, 32
    c_sizes = synth.uniform_sizes(n, 1000, 100000, seed_c)
    c_off = synth.offsets_from_sizes(c_sizes)
    rng = np.random.default_rng(seed_q)
    src = rng.integers(0, n, n_pl)
    bases = [synth.counter_ids(seed_c, int(c_off[r]), int(c_sizes[r]), D4) for r in src]
    planted, _ = synth.plant_near_duplicates(bases, D4, 0.75, 0.98, seed_q + 1)
    p_ids, p_off = synth.pack_sets(planted)
    q_sizes = np.concatenate([np.diff(p_off),
                              synth.uniform_sizes(nq - n_pl, 1000, 100000, seed_q + 2)])
    q_off = synth.offsets_from_sizes(q_sizes)
    q_ids = np.concatenate([p_ids, synth.counter_ids(seed_q + 3, 0, int(q_off[-1]) - len(p_ids),
                                                     D4)])
    with hoph.Plan(D4, K4, KG4, *AB4, perm_kind=hoph.HOPH_PERM_HASH61, seed=PERM_SEED, thr=T,
                   epsilon=EPS) as plan:
        planes = torch.empty((plan.G, n, KG4), dtype=torch.int32, device=dev)
        hoph.hoph_synth_sketch(plan.handle, seed_c, D4, to_dev(c_off, dev), n, planes)
        q = plan.sketch(to_dev(q_ids, dev), to_dev(q_off, dev), nq)
        plan.check()
        plan.set_exec(strategy=1, lanes_per_row=0, consumer_warps=16, stages=3)
        pairs, m, st = plan.query(hoph.HOPH_MODE_HOPH, q, nq, planes, n, stats=True)
        sample = np.unique(np.concatenate([np.random.default_rng(7).choice(n, 512, replace=False),
                                           pairs["row"].astype(np.int64), src]))
        got_rows = _device_rows(planes, sample, dev)
        got_q = planes_to_rows(q)
        G = plan.G
        del planes
        torch.cuda.empty_cache()
    lo = oc.layout(D4, K4, KG4, *AB4)
    hab = oc.hash_params(PERM_SEED)
    ids, offs = synth.pack_sets([synth.counter_ids(seed_c, int(c_off[r]), int(c_sizes[r]), D4)
                                 for r in sample])
    want_rows = oc.sketch(ids, offs, lo, D=D4, hash_ab=hab)
    want_q = oc.sketch(q_ids, q_off, lo, D=D4, hash_ab=hab)
    assert np.array_equal(got_q, want_q)
    assert np.array_equal(got_rows, want_rows)
    z = np.diff(lo[::KG4]).astype(np.uint64)
    want = oc.query("hoph", want_q, want_rows, KG4, T[0], T[1], EPS, z=z)["accepted"]
    want_set = {(int(a), int(sample[b]), int(g), int(mm)) for a, b, g, mm in want}
    got_set = {(int(p["query"]), int(p["row"]), int(p["groups"]), int(p["matches"]))
               for p in pairs}
    assert m == len(pairs) and m >= n_pl // 2
    assert got_set == want_set
    assert st.entering[0] == nq * n
    assert sum(st.accepted[g] for g in range(G)) == m
