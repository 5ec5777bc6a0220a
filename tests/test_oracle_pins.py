"""The CPU oracle pinned to the paper's worked examples, printed table,
closed forms, invariants and brute force.  No GPU."""
import json
import os
from fractions import Fraction
from itertools import permutations

import pytest

from oracle import hoph_ref as hr

GOLD = os.path.join(os.path.dirname(__file__), "golden")
E = hr.EMPTY


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _none_to_empty(v):
    if isinstance(v, list):
        return [_none_to_empty(x) for x in v]
    return E if v is None else v


IDENT = lambda x: x  # noqa: E731  (the worked examples use psi = identity)


# --- Sec. 3.2, OPH worked example -------------------------------------------

def test_oph_example_sketches_and_estimates():
    g = _gold("worked_examples.json")["oph_example"]
    lo, z = hr.layout(g["D"], g["k"], g["k"])
    sk = [hr.oph_sketch(S, IDENT, lo) for S in g["sets"]]
    assert sk == _none_to_empty(g["sketches"])
    # the stored value is the sample re-indexed to its offset inside the bin
    raw = _none_to_empty(g["samples_psi"])
    for s, r in zip(sk, raw):
        assert [E if v == E else v + lo[j] for j, v in enumerate(s)] == r
    assert hr.oph_estimate(sk[0], sk[1]) == Fraction(*g["estimate_12"])
    assert hr.oph_estimate(sk[0], sk[2], "either") == Fraction(*g["estimate_13_either"])
    assert hr.exact_jaccard(g["sets"][0], g["sets"][1]) == Fraction(*g["exact_12"])
    assert hr.exact_jaccard(g["sets"][0], g["sets"][2]) == Fraction(*g["exact_13"])
    # Eq. 5 (both empty) gives 1/4 for D1.D3: the printed 0.333 needs "either"
    assert hr.oph_estimate(sk[0], sk[2], "both") == Fraction(1, 4)


# --- Sec. 4.1, HOPH worked example ------------------------------------------

def test_hoph_example_layout_sketches_estimates():
    g = _gold("worked_examples.json")["hoph_example"]
    kg, G = g["k_group"], g["groups"]
    lo, z = hr.layout(g["D"], kg * G, kg, g["a"], g["b"])
    assert z == g["group_sizes"]
    sk = [hr.oph_sketch(S, IDENT, lo) for S in _gold("worked_examples.json")["oph_example"]["sets"]]
    printed = _none_to_empty(g["sketches_printed"])
    for s, p in zip(sk, printed):
        assert [s[i * kg:(i + 1) * kg] for i in range(G)] == p
    raw = _none_to_empty(g["samples_psi"])
    for s, r in zip(sk, raw):
        flat = [x for grp in r for x in grp]
        assert [E if v == E else v + lo[j] for j, v in enumerate(s)] == flat
    assert hr.hoph_estimate(sk[0], sk[1], kg, z) == Fraction(*g["estimate_12"])
    assert hr.hoph_estimate(sk[0], sk[1], kg, z, "either") == Fraction(*g["estimate_12"])
    assert hr.hoph_estimate(sk[0], sk[2], kg, z, "either") == Fraction(*g["estimate_13_either"])


def test_hoph_group_sizes_follow_ab_split():
    # 1:1 halves what remains; 1:2 gives a third; 2:1 two thirds (Sec. 4.1)
    assert hr.hoph_group_sizes(1 << 16, 4, 1, 1) == [32768, 16384, 8192, 8192]
    assert hr.hoph_group_sizes(1 << 20, 4, 1, 2) == [349525, 233017, 155344, 310690]
    assert hr.hoph_group_sizes(1 << 32, 4, 2, 1) == [2863311530, 954437177, 318145726,
                                                     159072863]
    lo, z = hr.layout(1 << 20, 256, 64, 1, 2)
    assert sum(z) == 1 << 20 and lo[0] == 0 and lo[-1] == 1 << 20
    assert all(lo[i] < lo[i + 1] for i in range(256))


# --- Table 2 and the small-probability limits ---------------------------------

def test_table2_binomial_tails():
    g = _gold("table2_binomial_k100_T0.6.json")
    bt = hr.BinomialTails(g["k_group"], Fraction(*g["T"]))
    for X, low, up in g["rows"]:
        for got, want in ((bt.lower(X), low), (bt.upper(X), up)):
            got = float(got)
            if want == 1.0:
                assert got == pytest.approx(1.0, abs=5e-10)
            else:
                assert got == pytest.approx(want, rel=2e-5, abs=5e-10), (X, got, want)


def test_tails_at_real_argument_use_ceiling():
    bt = hr.BinomialTails(100, Fraction(3, 5))
    assert bt.lower(Fraction(594, 10)) == bt.lower(60)       # P(X < 59.4) = P(X <= 59)
    assert bt.upper(Fraction(265, 4)) == bt.upper(67)        # P(X >= 66.25) = P(X >= 67)
    assert bt.lower(0) == 0 and bt.upper(0) == 1
    assert bt.lower(101) == 1 and bt.upper(101) == 0
    assert bt.upper(100) == Fraction(3, 5) ** 100           # closed form


def test_small_probability_limits():
    assert hr.small_probability_limits(100, Fraction(3, 5), 1e-4) == (79, 42)
    assert hr.small_probability_limits(64, Fraction(7, 10), 1e-4) == (58, 31)
    assert hr.small_probability_limits(32, Fraction(7, 10), 1e-4) == (32, 12)
    assert hr.small_probability_limits(128, Fraction(7, 10), 1e-4) == (109, 70)
    # eps = 0: nothing short of impossibility terminates
    assert hr.small_probability_limits(64, Fraction(7, 10), 0.0) == (65, 0)


# --- Example 1 (GOPH) and Example 2 (HOPH) ------------------------------------

def _pair_with_matches(kg, matches, groups):
    s = [0] * (kg * groups)
    t = [1] * (kg * groups)
    for g, m in enumerate(matches):
        for i in range(m):
            t[g * kg + i] = 0
    return s, t


def test_goph_example_1():
    g = _gold("worked_examples.json")["goph_example_1"]
    kg, n, T, eps = g["k_group"], g["n"], Fraction(*g["T"]), g["eps"]
    s, t = _pair_with_matches(kg, g["matches"], n)
    dec, groups, m = hr.goph_compare(s, t, kg, T, eps)
    assert (dec, groups, m) == (hr.REJECT, g["groups_compared"], sum(g["matches"]))
    # the first three groups alone leave the pair undecided (continue)
    s3, t3 = _pair_with_matches(kg, g["matches"][:3] + [60] * 7, n)
    assert hr.goph_compare(s3, t3, kg, T, eps)[1] > 3
    # F(x >= 85) = 5.0732E-08 is the event that ends it
    assert float(hr.BinomialTails(kg, T).upper(85)) == pytest.approx(5.0732e-08, rel=1e-4)


def test_hoph_example_2():
    g = _gold("worked_examples.json")["hoph_example_2"]
    kg, T, eps = g["k_group"], Fraction(*g["T"]), g["eps"]
    # two 1:1 groups of k'=100 bins: group 1 holds half the space (r = 1/2)
    lo, z = hr.layout(16 * kg, 2 * kg, kg, g["a"], g["b"])
    assert z[0] * 2 == sum(z)
    s, t = _pair_with_matches(kg, g["matches"] + [0], 2)
    for weighting in ("space", "literal"):
        dec, groups, _ = hr.hoph_compare(s, t, kg, z, T, eps, weighting=weighting,
                                         ab=(g["a"], g["b"]))
        assert (dec, groups) == (hr.REJECT, g["groups_compared"])
    # P_r * k' = 80 lies in the rejected upper tail: F(x >= 80) = 1.64119E-05
    assert float(hr.BinomialTails(kg, T).upper(80)) == pytest.approx(1.64119e-05, rel=1e-5)
    # with 43 matches P_r k' = 77, P(X >= 77) > eps: the pair continues
    s, t = _pair_with_matches(kg, [43, 0], 2)
    assert hr.hoph_compare(s, t, kg, z, T, eps)[1] == 2


# --- Exhaustive closed forms (Eq. 6-9) ----------------------------------------

@pytest.mark.parametrize("D,k,A,B", [(7, 3, [0, 1, 2, 4], [1, 2, 5, 6]),
                                     (6, 2, [0, 3], [0, 3, 4]),
                                     (6, 3, [1, 2, 3, 4, 5], [0, 5])])
def test_oph_unbiased_and_variance_exhaustive(D, k, A, B):
    """E[R] = Jaccard (Eq. 7) and the variance of Eq. 9, exactly, over all D!
    permutations; and MinWise's Pr[min equal] = Jaccard."""
    lo, _ = hr.layout(D, k, k)
    J = hr.exact_jaccard(A, B)
    n = 0
    s1 = s2 = einv = Fraction(0)
    mw = 0
    for p in permutations(range(D)):
        psi = p.__getitem__
        a = hr.oph_sketch(A, psi, lo)
        b = hr.oph_sketch(B, psi, lo)
        R = hr.oph_estimate(a, b)
        _, e, _ = hr.bin_counts(a, b)
        n += 1
        s1 += R
        s2 += R * R
        einv += Fraction(1, k - e)
        mw += hr.minwise_sketch(A, [psi]) == hr.minwise_sketch(B, [psi])
    Emean = s1 / n
    var = s2 / n - Emean * Emean
    g = len(set(A) | set(B))
    assert Emean == J
    assert var == J * (1 - J) * ((einv / n) * (1 + Fraction(1, g - 1)) - Fraction(1, g - 1))
    assert Fraction(mw, n) == J


def test_oph_unbiased_monte_carlo():
    """Mean of the estimator over many seeded permutations within 4 standard
    errors of the exact Jaccard (D = 64, k = 8)."""
    D, k = 64, 8
    lo, _ = hr.layout(D, k, k)
    A = list(range(0, 30))
    B = list(range(12, 40))
    J = float(hr.exact_jaccard(A, B))
    vals = []
    for seed in range(3000):
        perm = hr.permutation_table(D, seed)
        a = hr.oph_sketch(A, perm.__getitem__, lo)
        b = hr.oph_sketch(B, perm.__getitem__, lo)
        vals.append(float(hr.oph_estimate(a, b)))
    m = sum(vals) / len(vals)
    sd = (sum((v - m) ** 2 for v in vals) / (len(vals) - 1)) ** 0.5
    assert abs(m - J) < 4 * sd / len(vals) ** 0.5


# --- psi ----------------------------------------------------------------------

def test_splitmix64_published_vector():
    g = hr.SplitMix64(1234567)
    assert [g.next() for _ in range(5)] == [6457827717110365317, 3203168211198807973,
                                            9817491932198370423, 4593380528125082431,
                                            16408922859458223821]


def test_permutation_is_bijection_and_seeded():
    p = hr.permutation_table(1000, 1)
    assert sorted(p) == list(range(1000))
    assert p != list(range(1000))
    assert p == hr.permutation_table(1000, 1)
    assert p != hr.permutation_table(1000, 2)


def test_hash_perm_range():
    a, b = hr.hash_params(1)
    assert 1 <= a < hr.P61 and 0 <= b < hr.P61
    for x in (0, 1, 12345, (1 << 32) - 1):
        v = hr.hash_perm(x, a, b)
        assert 0 <= v < 1 << 32
        assert v == ((a * x + b) % hr.P61) >> 29


# --- Invariants of the decision rules -----------------------------------------

def _random_sketches(rng, n, lo, D, lo_size, hi_size):
    perm = hr.permutation_table(D, 5)
    out = []
    for _ in range(n):
        S = rng.sample(range(D), rng.randint(lo_size, hi_size))
        out.append((S, hr.oph_sketch(S, perm.__getitem__, lo)))
    return out


def test_identical_and_disjoint_invariants():
    import random
    rng = random.Random(3)
    D, k, kg = 256, 16, 4
    lo, z = hr.layout(D, k, kg, 1, 1)
    lo_e, _ = hr.layout(D, k, kg)
    perm = hr.permutation_table(D, 7)
    for _ in range(20):
        S = rng.sample(range(D), rng.randint(1, 60))
        rest = [x for x in range(D) if x not in set(S)]
        Tset = rng.sample(rest, rng.randint(1, 60))
        for lay in (lo, lo_e):
            a = hr.oph_sketch(S, perm.__getitem__, lay)
            b = hr.oph_sketch(Tset, perm.__getitem__, lay)
            m, e, x = hr.bin_counts(a, a)
            assert m == k - e and x == 0
            assert hr.bin_counts(a, b)[0] == 0       # psi is a bijection
        a = hr.oph_sketch(S, perm.__getitem__, lo)
        for T in (Fraction(1, 2), Fraction(7, 10), Fraction(1)):
            assert hr.hoph_compare(a, a, kg, z, T, 1e-4)[0] == hr.ACCEPT
            ae = hr.oph_sketch(S, perm.__getitem__, lo_e)
            assert hr.goph_compare(ae, ae, kg, T, 1e-4)[0] == hr.ACCEPT
            assert hr.oph_full_compare(ae, ae, T)[0] == hr.ACCEPT


def test_decision_reductions():
    """G = 1 makes GOPH plain OPH; eps = 0 makes early termination agree with
    the full scan; eps >= 1 ends every pair after one group."""
    import random
    rng = random.Random(11)
    D, k, kg = 512, 32, 8
    lo_e, _ = hr.layout(D, k, kg)
    lo_h, z = hr.layout(D, k, kg, 1, 1)
    perm = hr.permutation_table(D, 9)
    base = [rng.sample(range(D), rng.randint(5, 80)) for _ in range(12)]
    sets = base + [b[: len(b) // 2] + rng.sample(range(D), 5) for b in base]
    T = Fraction(1, 2)
    for A in sets:
        for B in sets:
            ae, be = (hr.oph_sketch(S, perm.__getitem__, lo_e) for S in (A, B))
            ah, bh = (hr.oph_sketch(S, perm.__getitem__, lo_h) for S in (A, B))
            full = hr.oph_full_compare(ae, be, T)[0]
            assert hr.goph_compare(ae, be, k, T, 1e-4)[0] == full          # G = 1
            assert hr.goph_compare(ae, be, kg, T, 0.0)[0] == full          # eps = 0
            hfull = hr.ACCEPT if (hr.hoph_estimate(ah, bh, kg, z) or 0) >= T else hr.REJECT
            assert hr.hoph_compare(ah, bh, kg, z, T, 0.0)[0] == hfull
            assert hr.goph_compare(ae, be, kg, T, 1.0)[1] == 1
            assert hr.hoph_compare(ah, bh, kg, z, T, 1.0)[1] == 1


def test_decision_monotone_in_matches():
    kg, G = 16, 4
    lo, z = hr.layout(1 << 12, kg * G, kg, 1, 2)
    T = Fraction(7, 10)
    rank = {hr.REJECT: 0, hr.CONTINUE: 1, hr.ACCEPT: 2}
    for rest in (0, 8, 16):
        prev_h = prev_g = -1
        for m in range(kg + 1):
            s, t = _pair_with_matches(kg, [m, rest, rest, rest], G)
            dh, gh, _ = hr.hoph_compare(s, t, kg, z, T, 1e-3)
            dg, gg, _ = hr.goph_compare(s, t, kg, T, 1e-3)
            # an early decision after group 1 never moves down as m grows
            vh = rank[dh] if gh == 1 else 1
            vg = rank[dg] if gg == 1 else 1
            assert vh >= prev_h and vg >= prev_g
            prev_h, prev_g = vh, vg


def test_precision_recall_definitions():
    p, r = hr.precision_recall({1, 2, 3, 4}, {2, 3, 5})
    assert (p, r) == (Fraction(2, 4), Fraction(2, 3))


# --- (a:b)HOPH with r != 1/2: Lemma 3 and Algorithm 2 pinned by the mathematics ---

@pytest.mark.parametrize("a,b", [(1, 2), (2, 1)])
@pytest.mark.parametrize("A,B", [([0, 1, 2, 4], [1, 2, 5, 6]),   # groups rarely empty
                                 ([0, 1], [1, 2]),                # union of 3: groups often empty
                                 ([3], [3, 6])])                  # one shared element of two
def test_hoph_space_weighted_estimator_unbiased_exhaustive(a, b, A, B):
    """Lemma 3 (Sec. 4.2) with the a:b space weights: within a group of equal
    bins a non-empty bin's minimum is a uniformly drawn element of the union
    given where the union's elements fall, so E[M_j / K_j] = J for every
    group, and the space-weighted mean over the groups that have a non-empty
    bin is exactly J whatever the weights.  Exhaustive over all 7!
    permutations for a 1:2 and a 2:1 layout (D = 7, k = 4, k' = 2; group
    sizes 2+5 and 4+3), including permutations that leave a group empty."""
    D, k, kg = 7, 4, 2
    lo, z = hr.layout(D, k, kg, a, b)
    assert z == ([2, 5] if (a, b) == (1, 2) else [4, 3])
    J = hr.exact_jaccard(A, B)
    total = Fraction(0)
    n = 0
    empty_groups = 0
    for p in permutations(range(D)):
        psi = p.__getitem__
        sa = hr.oph_sketch(A, psi, lo)
        sb = hr.oph_sketch(B, psi, lo)
        for g in range(2):
            if all(v == E for v in sa[g * kg:(g + 1) * kg] + sb[g * kg:(g + 1) * kg]):
                empty_groups += 1
        total += hr.hoph_estimate(sa, sb, kg, z)
        n += 1
    assert total / n == J
    if len(set(A) | set(B)) <= 3:
        assert empty_groups > 0  # the case where a group drops out of the weights is covered


def _expected_by_completion(s, t, kg, z, T, eps, bt):
    """The Algorithm 2 decision derived from Lemma 3's estimator alone.
    After l groups the remaining requirement is the smallest number c of
    matched bins that every remaining group (all bins non-empty) must reach
    for the final estimator to be >= T; the pair is already similar when the
    compared groups' own estimate exceeds T and P(X < c) <= eps, and already
    dissimilar otherwise when P(X >= c) <= eps (X ~ Bin(k', T); Def. 1).
    c is found by trying every completion, never from the P_r formula."""
    G = len(z)
    for l in range(1, G):
        pre_s, pre_t = s[:l * kg], t[:l * kg]
        done = hr.hoph_estimate(pre_s, pre_t, kg, z[:l])
        c_star = kg + 1
        for c in range(kg + 1):
            comp_s = pre_s + [0] * ((G - l) * kg)
            comp_t = pre_t + [0 if i % kg < c else 1 for i in range((G - l) * kg)]
            if hr.hoph_estimate(comp_s, comp_t, kg, z) >= T:
                c_star = c
                break
        if done is not None and done > T:
            if bt.lower(c_star) <= eps:
                return hr.ACCEPT, l
        else:
            if bt.upper(c_star) <= eps:
                return hr.REJECT, l
    est = hr.hoph_estimate(s, t, kg, z)
    return (hr.ACCEPT if est is not None and est >= T else hr.REJECT), G


@pytest.mark.parametrize("D,a,b", [(1 << 12, 1, 2), (1 << 12, 2, 1), (3000, 1, 3),
                                   (1 << 12, 1, 1)])
def test_hoph_space_rule_equals_the_requirement_from_lemma_3(D, a, b):
    """Every early accept / reject of the space-weighted (a:b)HOPH rule, for
    r != 1/2 as well as 1/2, equals the decision derived from completions of
    Lemma 3's estimator (above): catches a wrong remaining size Z_rem, a
    wrong group weight or a wrong tail.  Group states cover empty bins and
    whole empty groups."""
    import random
    rng = random.Random(17 + a * 7 + b)
    kg, G = 10, 4
    lo, z = hr.layout(D, kg * G, kg, a, b)
    seen = set()
    for T in (Fraction(7, 10), Fraction(1, 2), Fraction(3, 5)):
        bt = hr.BinomialTails(kg, T)
        for eps in (1e-4, 1e-2, 0.2, 0.5):
            for _ in range(150):
                s, t = [], []
                for g in range(G):
                    kind = rng.random()
                    for i in range(kg):
                        if kind < 0.1:                        # the whole group empty
                            s.append(E)
                            t.append(E)
                        elif rng.random() < 0.1:              # an empty bin on one side
                            s.append(E if rng.random() < 0.5 else 0)
                            t.append(0 if s[-1] == E and rng.random() < 0.5 else E)
                        else:
                            s.append(0)
                            t.append(0 if rng.random() < rng.choice((0.2, 0.6, 0.9)) else 1)
                got = hr.hoph_compare(s, t, kg, z, T, eps)
                want = _expected_by_completion(s, t, kg, z, T, eps, bt)
                assert got[:2] == want, (a, b, T, eps, s, t, got, want)
                seen.add(want)
    # early accepts, early rejects and full scans all occurred
    assert {d for d, l in seen if l < G} == {hr.ACCEPT, hr.REJECT}
    assert any(l == G for _, l in seen)


@pytest.mark.parametrize("a,b", [(1, 2), (2, 1)])
def test_decision_reductions_on_unequal_layouts(a, b):
    """On 1:2 and 2:1 layouts: eps = 0 makes the early-terminating HOPH rule
    decide exactly as Lemma 3's full estimator >= T, and eps >= 1 ends every
    pair after the first group."""
    import random
    rng = random.Random(23 + a)
    D, k, kg = 729, 32, 8
    lo, z = hr.layout(D, k, kg, a, b)
    perm = hr.permutation_table(D, 13)
    base = [rng.sample(range(D), rng.randint(3, 90)) for _ in range(12)]
    sets = base + [bs[: len(bs) // 2] + rng.sample(range(D), 4) for bs in base]
    for T in (Fraction(1, 2), Fraction(7, 10)):
        for A in sets:
            for B in sets:
                sa, sb = (hr.oph_sketch(S, perm.__getitem__, lo) for S in (A, B))
                est = hr.hoph_estimate(sa, sb, kg, z)
                full = hr.ACCEPT if est is not None and est >= T else hr.REJECT
                assert hr.hoph_compare(sa, sb, kg, z, T, 0.0)[0] == full
                assert hr.hoph_compare(sa, sb, kg, z, T, 1.0)[1] == 1
                assert hr.hoph_compare(sa, sb, kg, z, T, 2.5)[1] == 1


@pytest.mark.parametrize("a,b", [(1, 1), (1, 2), (2, 1), (3, 2)])
def test_literal_recursion_matches_its_closed_form(a, b):
    """Algorithm 2's printed recursion P_l = (P_{l-1} - (M_l/k') r^l) / r^l
    from P_0 = T unrolls to P_l = T / r^{s_l} - sum_j (M_j/k') / r^{s_l - s_j}
    with s_l = 1 + 2 + ... + l.  Every early decision of the oracle's literal
    weighting (Def. 1's tails at P_l k') must agree with that closed form, for
    r = a/(a+b) with a:b = 1:1, 1:2, 2:1, 3:2 and random match counts over
    four groups (no empty bins, so K = k')."""
    import random
    rng = random.Random(5 + 10 * a + b)
    kg, G = 8, 4
    lo, z = hr.layout(4096, kg * G, kg, a, b)
    r = Fraction(a, a + b)
    for T in (Fraction(7, 10), Fraction(1, 2)):
        bt = hr.BinomialTails(kg, T)
        for eps in (1e-3, 0.05, 0.3):
            for _ in range(60):
                ms = [rng.randint(0, kg) for _ in range(G)]
                s_, t_ = _pair_with_matches(kg, ms, G)
                got = hr.hoph_compare(s_, t_, kg, z, T, eps, weighting="literal", ab=(a, b))
                want = None
                for l in range(1, G):
                    sl = l * (l + 1) // 2
                    P = T / r ** sl - sum(Fraction(ms[j - 1], kg) / r ** (sl - j * (j + 1) // 2)
                                          for j in range(1, l + 1))
                    if P < T and bt.lower(P * kg) <= eps:
                        want = (hr.ACCEPT, l)
                        break
                    if P >= T and bt.upper(P * kg) <= eps:
                        want = (hr.REJECT, l)
                        break
                if want is None:  # all groups: the space-weighted estimator (Lemma 3)
                    est = hr.hoph_estimate(s_, t_, kg, z)
                    want = ((hr.ACCEPT if est is not None and est >= T else hr.REJECT), G)
                assert got[:2] == want, (a, b, T, eps, ms, got, want)
