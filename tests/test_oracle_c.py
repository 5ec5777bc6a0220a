"""The scalable C oracle agrees with the exact Python oracle (which the pins
tie to the paper).  No GPU."""
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import hoph_ref as hr
from oracle import oracle_c as oc
from paper_1805_11254_gb300 import synth


def test_permutation_tables_equal():
    for D, seed in ((1, 3), (2, 1), (1000, 1), (1 << 16, 1), (4097, 77)):
        assert oc.permutation(D, seed).tolist() == hr.permutation_table(D, seed)


def test_hash_params_and_values_equal():
    a, b = oc.hash_params(1)
    assert (a, b) == hr.hash_params(1)
    lib = oc.load()
    for x in (0, 1, 2, 99, 123456789, (1 << 32) - 1):
        assert lib.or_hash_psi(x, a, b) == hr.hash_perm(x, a, b)


@pytest.mark.parametrize("D,k,kg,a,b", [(16, 4, 4, 0, 0), (16, 6, 2, 1, 1), (1 << 16, 128, 32, 1, 1),
                                        (1 << 20, 256, 64, 1, 2), (1 << 32, 512, 128, 2, 1),
                                        (1000, 12, 3, 0, 0), (12345, 40, 8, 3, 5)])
def test_layouts_equal(D, k, kg, a, b):
    assert oc.layout(D, k, kg, a, b).tolist() == hr.layout(D, k, kg, a, b)[0]


def test_tails_match_exact():
    for kg, tn, td in ((100, 6, 10), (64, 7, 10), (32, 1, 3), (128, 7, 10), (7, 1, 1), (5, 0, 1)):
        low, up = oc.tails(kg, tn, td)
        bt = hr.BinomialTails(kg, Fraction(tn, td))
        for m in range(kg + 2):
            assert low[m] == pytest.approx(float(bt.low[m]), rel=1e-12, abs=1e-300)
            assert up[m] == pytest.approx(float(bt.up[m]), rel=1e-12, abs=1e-300)


def _sets(rng, n, D, lo, hi, empty_every=0):
    sets = []
    for i in range(n):
        if empty_every and i % empty_every == 0:
            sets.append([])
        else:
            sets.append(rng.sample(range(D), rng.randint(lo, hi)))
    return sets


def test_sketches_equal_table_and_hash():
    rng = random.Random(5)
    D, k, kg = 4096, 32, 8
    perm = hr.permutation_table(D, 1)
    sets = _sets(rng, 40, D, 1, 200, empty_every=13)
    ids, off = synth.pack_sets(sets)
    for a, b in ((0, 0), (1, 1), (1, 2), (2, 1)):
        lo, _ = hr.layout(D, k, kg, a, b)
        got = oc.sketch(ids, off, lo, perm=np.asarray(perm, dtype=np.uint32))
        want = [hr.oph_sketch(S, perm.__getitem__, lo) for S in sets]
        assert got.tolist() == want
    ha, hb = hr.hash_params(1)
    lo, _ = hr.layout(1 << 32, 64, 16, 2, 1)
    ids32 = np.asarray([rng.getrandbits(32) for _ in range(3000)], dtype=np.uint32)
    off32 = np.asarray([0, 1000, 1000, 3000], dtype=np.int64)
    got = oc.sketch(ids32, off32, lo, D=1 << 32, hash_ab=(ha, hb))
    for i in range(3):
        S = ids32[off32[i]:off32[i + 1]].tolist()
        assert got[i].tolist() == hr.oph_sketch(S, lambda x: hr.hash_perm(x, ha, hb), lo)


def test_minwise_equal():
    rng = random.Random(6)
    D, k = 512, 8
    perms = [hr.permutation_table(D, 1 + t) for t in range(k)]
    sets = _sets(rng, 20, D, 1, 50, empty_every=7)
    ids, off = synth.pack_sets(sets)
    got = oc.minwise(ids, off, np.asarray(perms, dtype=np.uint32))
    want = [hr.minwise_sketch(S, [p.__getitem__ for p in perms]) for S in sets]
    assert got.tolist() == want


@pytest.mark.parametrize("rule", ["both", "either", "none"])
@pytest.mark.parametrize("eps", [0.0, 1e-4, 0.05, 1.0])
def test_query_decisions_equal(rule, eps):
    rng = random.Random(hash((rule, eps)) & 0xFFFF)
    D, kg, G = 2048, 8, 4
    k = kg * G
    perm = hr.permutation_table(D, 3)
    base = _sets(rng, 10, D, 1, 120, empty_every=9)
    sets = base + [b[: max(1, len(b) * 3 // 4)] + rng.sample(range(D), 3) for b in base if b]
    T = Fraction(3, 5)
    for mode, ab in (("goph", (0, 0)), ("hoph", (1, 1)), ("hoph", (1, 2)), ("hoph", (2, 1)),
                     ("oph_full", (0, 0))):
        lo, z = hr.layout(D, k, kg, *ab)
        sk = np.asarray([hr.oph_sketch(S, perm.__getitem__, lo) for S in sets], dtype=np.uint32)
        res = oc.query(mode, sk, sk, kg, 3, 5, eps, rule=rule, z=np.asarray(z), per_pair=True)
        for i in range(len(sets)):
            for j in range(len(sets)):
                s, t = sk[i].tolist(), sk[j].tolist()
                if mode == "goph":
                    want = hr.goph_compare(s, t, kg, T, eps, rule)
                elif mode == "hoph":
                    want = hr.hoph_compare(s, t, kg, z, T, eps, rule)
                else:
                    want = hr.oph_full_compare(s, t, T, rule)
                got = (int(res["dec"][i, j]), int(res["groups"][i, j]), int(res["msum"][i, j]))
                assert got == want, (mode, ab, i, j)
        acc = [(int(q), int(r)) for q, r, _, _ in res["accepted"]]
        assert acc == sorted((i, j) for i in range(len(sets)) for j in range(len(sets))
                             if res["dec"][i, j] == hr.ACCEPT)


@pytest.mark.parametrize("eps", [0.0, 1e-4, 0.05, 1.0])
def test_literal_recursion_decisions_equal(eps):
    """Algorithm 2 as printed (weighting 'literal'): the C oracle's reduced
    fractions against the Fraction reference, over (a:b) splits whose r is
    1/2, 1/3, 2/3 and 3/4."""
    rng = random.Random(int(eps * 1e6) + 7)
    D, kg, G = 4096, 16, 4
    k = kg * G
    perm = hr.permutation_table(D, 5)
    base = _sets(rng, 10, D, 1, 300, empty_every=9)
    sets = base + [b[: max(1, len(b) * 4 // 5)] + rng.sample(range(D), 2) for b in base if b]
    T = Fraction(3, 5)
    for ab in ((1, 1), (1, 2), (2, 1), (3, 1)):
        lo, z = hr.layout(D, k, kg, *ab)
        sk = np.asarray([hr.oph_sketch(S, perm.__getitem__, lo) for S in sets], dtype=np.uint32)
        res = oc.query("hoph", sk, sk, kg, 3, 5, eps, z=np.asarray(z), per_pair=True,
                       weighting="literal", ab=ab)
        seen = set()
        for i in range(len(sets)):
            for j in range(len(sets)):
                s, t = sk[i].tolist(), sk[j].tolist()
                want = hr.hoph_compare(s, t, kg, z, T, eps, weighting="literal", ab=ab)
                got = (int(res["dec"][i, j]), int(res["groups"][i, j]), int(res["msum"][i, j]))
                assert got == want, (ab, i, j)
                seen.add(want[:2])
        if eps == 1e-4:  # the cases reach more than the first group
            assert any(g > 1 for _, g in seen)


def test_minwise_decisions_equal():
    rng = random.Random(8)
    D, k = 256, 16
    perms = [hr.permutation_table(D, 1 + t) for t in range(k)]
    sets = _sets(rng, 15, D, 1, 60, empty_every=6)
    sk = np.asarray([hr.minwise_sketch(S, [p.__getitem__ for p in perms]) for S in sets],
                    dtype=np.uint32)
    res = oc.query("minwise_full", sk, sk, k, 7, 10, 1e-4, per_pair=True)
    for i in range(len(sets)):
        for j in range(len(sets)):
            want = hr.minwise_compare(sk[i].tolist(), sk[j].tolist(), Fraction(7, 10))
            assert (int(res["dec"][i, j]), int(res["msum"][i, j])) == (want[0], want[2])


def test_pair_counts_and_jaccard():
    rng = random.Random(9)
    D, kg, G = 1024, 4, 3
    lo, _ = hr.layout(D, kg * G, kg, 1, 1)
    perm = hr.permutation_table(D, 2)
    sets = _sets(rng, 8, D, 0, 40)
    sk = np.asarray([hr.oph_sketch(S, perm.__getitem__, lo) for S in sets], dtype=np.uint32)
    cnt = oc.pair_counts(sk, sk, kg)
    for i in range(8):
        for j in range(8):
            for g in range(G):
                want = hr.bin_counts(sk[i, g * kg:(g + 1) * kg].tolist(),
                                     sk[j, g * kg:(g + 1) * kg].tolist())
                assert tuple(int(v) for v in cnt[i, j, g]) == want
    ids, off = synth.pack_sets([S + S[:3] for S in sets])     # duplicates are ignored
    pa = np.repeat(np.arange(8), 8)
    pb = np.tile(np.arange(8), 8)
    inter, uni = oc.jaccard_pairs(ids, off, ids, off, pa, pb)
    for n, (i, j) in enumerate(zip(pa, pb)):
        A, B = set(sets[i]), set(sets[j])
        assert (inter[n], uni[n]) == (len(A & B), len(A | B))
