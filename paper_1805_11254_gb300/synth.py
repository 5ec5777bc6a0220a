"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds random-number generation only (no sketching, no
comparison arithmetic).  Tests and the benchmark feed its arrays both to the
CUDA library and to the CPU oracle.

Sets are ID lists over a vocabulary {0..D-1}: CSR form, ``ids`` (uint32)
plus ``offsets`` (int64, n+1 entries).

Two kinds of generator:

* numpy ``Generator(PCG64(seed))`` for small, exact workloads (distinct IDs,
  planted near duplicates);
* a counter-based generator for the large collections: element e of a
  stream with seed s takes the e-th output of SplitMix64 seeded with s,
  ``mix(s + (e+1) * 0x9E3779B97F4A7C15)``, mapped to [0, D) by a
  multiply-shift of its top 32 bits.  The same definition is implemented on
  the device (``hoph_synth_ids``) so a multi-GB collection can be generated
  in HBM and any one of its sets regenerated here, on the host.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix_at(seed, counters):
    """The (counter+1)-th SplitMix64 output of the stream seeded with ``seed``,
    vectorised over ``counters`` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def counter_ids(seed, start, count, D):
    """IDs of global elements start..start+count-1: ((h >> 32) * D) >> 32."""
    e = np.arange(start, start + count, dtype=np.uint64)
    h = splitmix_at(seed, e) >> np.uint64(32)
    with np.errstate(over="ignore"):
        if D == 1 << 32:
            return h.astype(np.uint32)
        return ((h * np.uint64(D)) >> np.uint64(32)).astype(np.uint32)


def counter_uniform01(seed, start, count):
    """Doubles in [0, 1): (h >> 11) * 2^-53 (exact in binary64)."""
    e = np.arange(start, start + count, dtype=np.uint64)
    h = splitmix_at(seed, e) >> np.uint64(11)
    return h.astype(np.float64) * (1.0 / 9007199254740992.0)


def zipf_cdf(D, s):
    """CDF table of a Zipf(s) law over ranks 1..D (float64, last entry 1)."""
    w = np.arange(1, D + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    c /= c[-1]
    c[-1] = 1.0
    return c


def counter_zipf_ids(seed, start, count, cdf):
    """Zipf IDs (rank - 1) by inverse CDF of counter uniforms: the first index
    i with u < cdf[i]."""
    u = counter_uniform01(seed, start, count)
    return np.searchsorted(cdf, u, side="right").astype(np.uint32)


def offsets_from_sizes(sizes):
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def lognormal_sizes(n, median, sigma, lo, hi, seed):
    """Set sizes ~ lognormal(ln median, sigma), rounded, clipped to [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = np.rint(rng.lognormal(np.log(median), sigma, n))
    return np.clip(s, lo, hi).astype(np.int64)


def uniform_sizes(n, lo, hi, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, n, dtype=np.int64)


def distinct_uniform_sets(sizes, D, seed):
    """Sets of distinct IDs drawn uniformly from {0..D-1}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    off = offsets_from_sizes(sizes)
    ids = np.empty(int(off[-1]), dtype=np.uint32)
    for i, s in enumerate(sizes):
        s = int(s)
        if s * 4 < D:
            got = np.unique(rng.integers(0, D, s + s // 8 + 8, dtype=np.int64))
            while len(got) < s:
                got = np.unique(np.concatenate([got, rng.integers(0, D, s, dtype=np.int64)]))
            got = rng.permutation(got)[:s]
        else:
            got = rng.choice(D, s, replace=False)
        ids[off[i]:off[i + 1]] = got
    return ids, off


def plant_near_duplicates(src_sets, D, j_lo, j_hi, seed):
    """Near duplicates of given sets: for a set of s distinct IDs and a target
    Jaccard J ~ U[j_lo, j_hi], t = round(s(1-J)/(1+J)) of its IDs are swapped
    for fresh IDs not in it (so J = (s-t)/(s+t)).  Returns the new sets and the
    drawn targets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    targets = []
    for base in src_sets:
        base = np.unique(np.asarray(base, dtype=np.int64))
        s = len(base)
        J = rng.uniform(j_lo, j_hi)
        t = int(round(s * (1 - J) / (1 + J)))
        t = min(t, s)
        keep = rng.permutation(base)[: s - t]
        have = set(base.tolist())
        fresh = []
        while len(fresh) < t:
            x = int(rng.integers(0, D))
            if x not in have:
                have.add(x)
                fresh.append(x)
        new = np.concatenate([keep, np.asarray(fresh, dtype=np.int64)])
        out.append(rng.permutation(new).astype(np.uint32))
        targets.append(J)
    return out, np.asarray(targets)


def pack_sets(sets):
    sizes = np.asarray([len(s) for s in sets], dtype=np.int64)
    off = offsets_from_sizes(sizes)
    ids = np.concatenate([np.asarray(s, dtype=np.uint32) for s in sets]) if len(sets) else \
        np.zeros(0, dtype=np.uint32)
    return ids, off


def unpack(ids, off, i):
    return ids[off[i]:off[i + 1]]


# ---------------------------------------------------------------------------
# The workloads
# ---------------------------------------------------------------------------

def small_parity_workload(n=5000, D=1 << 16, size_lo=50, size_hi=500, n_queries=50,
                          j_lo=0.3, j_hi=0.95, seed_coll=11, seed_q=12, seed_plant=13):
    """N sets of U[size_lo, size_hi] distinct uniform IDs over D, plus
    n_queries planted near duplicates of random collection sets at Jaccard
    ~ U[j_lo, j_hi]."""
    sizes = uniform_sizes(n, size_lo, size_hi, seed_coll)
    ids, off = distinct_uniform_sets(sizes, D, seed_coll + 1000)
    rng = np.random.Generator(np.random.PCG64(seed_q))
    src = rng.integers(0, n, n_queries)
    qsets, targets = plant_near_duplicates([unpack(ids, off, int(r)) for r in src], D,
                                           j_lo, j_hi, seed_plant)
    q_ids, q_off = pack_sets(qsets)
    return dict(ids=ids, off=off, q_ids=q_ids, q_off=q_off, src=src, targets=targets, D=D)


def counter_collection_sizes(n, seed, median=300, sigma=1.0, lo=10, hi=20000):
    return lognormal_sizes(n, median, sigma, lo, hi, seed)


def query_batch(n_queries, frac_planted, D, coll_seed, coll_off, j_lo, j_hi, seed_q,
                seed_plant, median=300, sigma=1.0, lo=10, hi=20000):
    """A batch of queries against a counter-generated collection (uniform IDs
    over D): a fraction are near duplicates of random collection rows, the
    rest fresh random sets of the same size law."""
    rng = np.random.Generator(np.random.PCG64(seed_q))
    n_rows = len(coll_off) - 1
    n_pl = int(round(n_queries * frac_planted))
    src = rng.integers(0, n_rows, n_pl)
    bases = [counter_ids(coll_seed, int(coll_off[r]), int(coll_off[r + 1] - coll_off[r]), D)
             for r in src]
    planted, targets = plant_near_duplicates(bases, D, j_lo, j_hi, seed_plant)
    fresh_sizes = lognormal_sizes(n_queries - n_pl, median, sigma, lo, hi, seed_q + 1)
    f_ids, f_off = distinct_uniform_sets(fresh_sizes, D, seed_q + 2)
    sets = planted + [unpack(f_ids, f_off, i) for i in range(len(fresh_sizes))]
    order = rng.permutation(n_queries)
    sets = [sets[i] for i in order]
    is_planted = np.zeros(n_queries, dtype=bool)
    src_of = np.full(n_queries, -1, dtype=np.int64)
    for new_pos, old in enumerate(order):
        if old < n_pl:
            is_planted[new_pos] = True
            src_of[new_pos] = src[old]
    q_ids, q_off = pack_sets(sets)
    return dict(q_ids=q_ids, q_off=q_off, src=src_of, planted=is_planted)
