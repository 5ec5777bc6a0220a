"""The input recipe (no GPU): the seeded generators produce the shapes the
workloads state - counter streams that can be regenerated piecewise, the
lognormal size law with its clipping, the Zipf(1.1) law, distinct uniform
sets, and planted near duplicates at their drawn Jaccard."""
import numpy as np

from paper_1805_11254_gb300 import synth


def test_counter_stream_regenerates_any_slice():
    seed, D = 11, 1 << 20
    whole = synth.counter_ids(seed, 1000, 5000, D)
    parts = np.concatenate([synth.counter_ids(seed, 1000, 1234, D),
                            synth.counter_ids(seed, 2234, 3766, D)])
    assert np.array_equal(whole, parts)
    assert whole.dtype == np.uint32 and whole.max() < D
    assert not np.array_equal(whole, synth.counter_ids(seed + 1, 1000, 5000, D))


def test_counter_ids_are_uniform_over_the_vocabulary():
    D = 1 << 8
    ids = synth.counter_ids(3, 0, 256 * 4000, D)
    counts = np.bincount(ids, minlength=D)
    chi2 = float(((counts - 4000.0) ** 2 / 4000.0).sum())
    assert chi2 < 2 * D  # 255 degrees of freedom: mean 255, sd ~23
    full = synth.counter_ids(3, 0, 1000, 1 << 32)
    assert full.dtype == np.uint32 and len(np.unique(full)) == 1000


def test_counter_uniforms_lie_in_the_unit_interval():
    u = synth.counter_uniform01(5, 0, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005


def test_lognormal_sizes_follow_the_stated_law():
    s = synth.lognormal_sizes(200000, 300, 1.0, 10, 20000, 21)
    assert s.min() >= 10 and s.max() <= 20000
    assert abs(np.median(s) - 300) < 6
    # ln-sizes have sigma ~1 away from the clipped tails
    ln = np.log(s[(s > 30) & (s < 3000)])
    assert 0.7 < ln.std() < 1.0
    assert np.array_equal(s, synth.lognormal_sizes(200000, 300, 1.0, 10, 20000, 21))


def test_zipf_law_table_and_draws():
    D, a = 1 << 12, 1.1
    cdf = synth.zipf_cdf(D, a)
    assert np.all(np.diff(cdf) > 0) and cdf[-1] == 1.0
    h = (np.arange(1, D + 1, dtype=np.float64) ** -a).sum()
    assert abs(cdf[0] - 1.0 / h) < 1e-12
    ids = synth.counter_zipf_ids(21, 0, 400000, cdf)
    assert ids.max() < D
    f = np.bincount(ids, minlength=D) / len(ids)
    assert abs(f[0] - 1.0 / h) < 0.004
    assert abs(f[0] / f[1] - 2 ** a) < 0.08  # P(rank 1) / P(rank 2) = 2^a


def test_distinct_uniform_sets_have_their_sizes_and_no_repeats():
    sizes = synth.uniform_sizes(300, 1, 700, 4)
    for D in (1 << 10, 1 << 16):
        ids, off = synth.distinct_uniform_sets(np.minimum(sizes, D), D, 9)
        for i in range(len(sizes)):
            s = synth.unpack(ids, off, i)
            assert len(s) == min(sizes[i], D) and len(np.unique(s)) == len(s)
            assert s.max() < D


def test_planted_near_duplicates_have_their_drawn_jaccard():
    D = 1 << 16
    bases = [synth.counter_ids(1, 1000 * i, 200 + 37 * i, D) for i in range(40)]
    planted, targets = synth.plant_near_duplicates(bases, D, 0.3, 0.95, 13)
    assert len(planted) == len(bases)
    for b, p, J in zip(bases, planted, targets):
        b = set(np.unique(b).tolist())
        p_list = p.tolist()
        assert len(set(p_list)) == len(p_list) == len(b)  # same size, distinct
        inter = len(b & set(p_list))
        s = len(b)
        t = s - inter
        assert t == min(int(round(s * (1 - J) / (1 + J))), s)
        jac = inter / (2 * s - inter)
        assert abs(jac - J) < 2.0 / s + 1e-9  # one swap moves J by < 2/s
        assert 0.3 <= J <= 0.95


def test_pack_and_unpack_round_trip():
    sets = [np.array([3, 1, 2], dtype=np.uint32), np.zeros(0, dtype=np.uint32),
            np.array([7], dtype=np.uint32)]
    ids, off = synth.pack_sets(sets)
    assert off.tolist() == [0, 3, 3, 4]
    for i, s in enumerate(sets):
        assert np.array_equal(synth.unpack(ids, off, i), s)
