"""Exact CPU oracle for OPH, GOPH, (a:b)HOPH and MinWise.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may use it.  It shares no code with the CUDA library.

Everything here is plain Python on exact integers and ``fractions.Fraction``:
slow, and meant to be read against the paper (Zhang et al., "Hierarchical One
Permutation Hashing: Efficient Multimedia Near Duplicate Detection",
arXiv 1805.11254).  Section / equation / algorithm numbers below are the
paper's.

Readings taken where the paper is garbled or silent:

* near duplicate means Jaccard >= T (Sec. 3.1 prints "<", the rest of the
  paper tests ">=");
* the vocabulary of the worked examples is {0..15} (16 values);
* the stored per-bin value is (min psi-value in the bin) - (bin lower bound),
  the "smallest possible representation" of Sec. 3.2 / 4.1;
* F(x) has two tails: lower P(X < m) and upper P(X >= m), evaluated at
  ceil(m) for a real m (Table 2 pins both);
* a pair terminates iff the relevant tail is <= eps (Definition 1);
* after l groups GOPH uses M_ra = (T*(K_c + (n-l)k') - M_c)/(n-l) with l the
  number of groups already compared (Example 1), pooled over non-empty bins;
* HOPH uses the space-weighted remaining requirement
  P_r = (T*(Z_done + Z_rem) - S)/Z_rem, S = sum z_j M_j / K_j (Lemma 3's
  estimator with the a:b group sizes as weights); ``weighting='literal'``
  keeps Algorithm 2's r^l recursion instead;
* when every group has been compared the pair is accepted iff the full
  estimator (Eq. 6 for OPH/GOPH, Lemma 3 for HOPH) is >= T;
* empty bins: ``rule='both'`` drops bins empty in both sketches (Eq. 5, the
  default), ``'either'`` drops bins empty in either (reproduces the worked
  examples' 0.333 and 0.375), ``'none'`` keeps all k' bins (Algorithms 1/2
  taken literally).
"""

from bisect import bisect_right
from fractions import Fraction
from functools import lru_cache
from math import comb

EMPTY = 0xFFFFFFFF          # the empty-bin marker (the paper's circled-times)
MASK64 = (1 << 64) - 1
P61 = (1 << 61) - 1         # Mersenne prime of the 2-universal hash

ACCEPT, REJECT, CONTINUE = 1, 2, 0


# ---------------------------------------------------------------------------
# psi: the single random permutation (Sec. 3.2)
# ---------------------------------------------------------------------------

class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the seeded PRNG that
    drives the Fisher-Yates shuffle and the hash parameters."""

    def __init__(self, seed):
        self.state = seed & MASK64

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def permutation_table(D, seed):
    """psi: V -> V (Sec. 3.2) as an explicit table over V = {0..D-1}.

    Fisher-Yates from the identity: for i = D-1 down to 1, j = next() mod
    (i+1), swap entries i and j.
    """
    perm = list(range(D))
    rng = SplitMix64(seed)
    for i in range(D - 1, 0, -1):
        j = rng.next() % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def hash_params(seed):
    """(a, b) of the 2-universal hash used when D is too large for a table:
    a = 1 + next() mod (p-1), b = next() mod p, p = 2^61 - 1."""
    rng = SplitMix64(seed)
    a = 1 + rng.next() % (P61 - 1)
    b = rng.next() % P61
    return a, b


def hash_perm(x, a, b):
    """psi(x) = ((a*x + b) mod (2^61-1)) >> 29: a 32-bit value (not a
    bijection; stands in for psi when V = 2^32)."""
    return ((a * x + b) % P61) >> 29


# ---------------------------------------------------------------------------
# Bin layout (Sec. 3.2 for OPH/GOPH, Sec. 4.1 for (a:b)HOPH)
# ---------------------------------------------------------------------------

def _ceil_div(a, b):
    return -((-a) // b)


def hoph_group_sizes(D, G, a, b):
    """(a:b)HOPH space division (Sec. 4.1): each split gives the permutation
    group a/(a+b) of what remains (floored); the last group takes the rest."""
    sizes = []
    rem = D
    for _ in range(G - 1):
        zg = rem * a // (a + b)
        sizes.append(zg)
        rem -= zg
    sizes.append(rem)
    return sizes


def layout(D, k, kg, a=0, b=0):
    """Return (lo, z): bin lower bounds lo[0..k] (lo[k] = D) in psi-space and
    the group sizes z[0..G-1].  Bin j holds psi-values in [lo[j], lo[j+1]);
    group g is bins [g*kg, (g+1)*kg).

    a = b = 0: OPH/GOPH, the space split evenly into k bins (Sec. 3.2),
    lo[j] = ceil(j*D/k), then grouped kg bins at a time (Sec. 3.3).
    Otherwise (a:b)HOPH: group sizes from ``hoph_group_sizes`` and each group
    split evenly into kg bins (Sec. 4.1).
    """
    if k % kg:
        raise ValueError("k must be a multiple of k'")
    G = k // kg
    if a == 0 and b == 0:
        if D < k:
            raise ValueError("D < k")
        lo = [_ceil_div(j * D, k) for j in range(k + 1)]
    else:
        zs = hoph_group_sizes(D, G, a, b)
        if min(zs) < kg:
            raise ValueError("a group smaller than k' bins")
        lo = []
        start = 0
        for zg in zs:
            for i in range(kg):
                lo.append(start + _ceil_div(i * zg, kg))
            start += zg
        lo.append(D)
    z = [lo[(g + 1) * kg] - lo[g * kg] for g in range(G)]
    return lo, z


# ---------------------------------------------------------------------------
# Sketches
# ---------------------------------------------------------------------------

def oph_sketch(S, psi, lo):
    """OPH / HOPH sketch (Sec. 3.2, Sec. 4.1): per bin the smallest psi-value
    of the set that falls in it, re-indexed to its offset inside the bin;
    EMPTY when no element of the set falls in the bin."""
    k = len(lo) - 1
    sk = [EMPTY] * k
    for x in S:
        p = psi(x)
        j = bisect_right(lo, p) - 1
        v = p - lo[j]
        if v < sk[j]:
            sk[j] = v
    return sk


def minwise_sketch(S, psis):
    """MinWise (Sec. 1): the minimum of the set under each of k independent
    permutations; EMPTY for the empty set."""
    return [min((psi(x) for x in S), default=EMPTY) for psi in psis]


# ---------------------------------------------------------------------------
# Per-bin indicators and group counts (Eq. 2-5)
# ---------------------------------------------------------------------------

def bin_counts(s, t):
    """(matched, both-empty, exactly-one-empty) over aligned bins.

    A bin matches when both samples are non-empty and equal (Eq. 4); it is an
    empty bin when both are EMPTY (Eq. 5)."""
    m = e = x = 0
    for u, v in zip(s, t):
        if u == EMPTY and v == EMPTY:
            e += 1
        elif u == EMPTY or v == EMPTY:
            x += 1
        elif u == v:
            m += 1
    return m, e, x


def effective_bins(kg, e, x, rule):
    """Number of bins that count in the denominator under each empty rule."""
    if rule == "both":
        return kg - e
    if rule == "either":
        return kg - e - x
    if rule == "none":
        return kg
    raise ValueError(rule)


# ---------------------------------------------------------------------------
# Binomial tails and the small-probability event (Eq. 10-11, Definition 1)
# ---------------------------------------------------------------------------

class BinomialTails:
    """X ~ Bin(k', T).  lower(m) = P(X < m), upper(m) = P(X >= m), exact.

    A real argument m is evaluated at ceil(m) (X is integer-valued), so
    lower(59.4) = P(X <= 59) and upper(66.25) = P(X >= 67)."""

    def __init__(self, kg, T):
        self.kg = kg
        T = Fraction(T)
        pmf = [comb(kg, j) * T ** j * (1 - T) ** (kg - j) for j in range(kg + 1)]
        self.low = [Fraction(0)] * (kg + 2)     # low[m] = P(X < m), m = 0..kg+1
        for m in range(1, kg + 2):
            self.low[m] = self.low[m - 1] + pmf[m - 1]
        self.up = [Fraction(0)] * (kg + 2)      # up[m] = P(X >= m)
        for m in range(kg, -1, -1):
            self.up[m] = self.up[m + 1] + pmf[m]

    def _index(self, m):
        c = m if isinstance(m, int) else _ceil_fraction(Fraction(m))
        return c

    def lower(self, m):
        c = self._index(m)
        if c <= 0:
            return Fraction(0)
        if c > self.kg:
            return Fraction(1)
        return self.low[c]

    def upper(self, m):
        c = self._index(m)
        if c <= 0:
            return Fraction(1)
        if c > self.kg:
            return Fraction(0)
        return self.up[c]


def _ceil_fraction(f):
    return -((-f.numerator) // f.denominator)


@lru_cache(maxsize=64)
def _tails_cached(kg, T):
    return BinomialTails(kg, T)


def small_probability_limits(kg, T, eps):
    """U = min{j : P(X >= j) <= eps}, L = max{j : P(X < j) <= eps}.

    Not used by the decisions below (they evaluate the tails directly); kept
    so tests can compare against the library's precomputed limits."""
    bt = _tails_cached(kg, Fraction(T))
    e = Fraction(eps)
    U = next(j for j in range(kg + 2) if bt.up[j] <= e)
    L = max(j for j in range(kg + 2) if bt.low[j] <= e)
    return U, L


# ---------------------------------------------------------------------------
# Comparison rules
# ---------------------------------------------------------------------------

def _group(s, g, kg):
    return s[g * kg:(g + 1) * kg]


def goph_compare(s, t, kg, T, eps, rule="both"):
    """GOPH comparison (Algorithm 1, Sec. 3.3) of two k-bin sketches grouped
    into n = k/k' groups.  Returns (decision, groups compared, matched bins).

    After l groups (l < n): M_ra = (T*(K_c + (n-l)k') - M_c)/(n-l) and
    M_a = T k'.  If M_ra < M_a and P(X < M_ra) <= eps the pair is similar;
    if M_ra >= M_a and P(X >= M_ra) <= eps it is not; otherwise compare the
    next group.  After all n groups: similar iff K_c > 0 and M_c >= T K_c
    (Eq. 6)."""
    T = Fraction(T)
    eps = Fraction(eps)
    n = len(s) // kg
    bt = BinomialTails(kg, T)
    Mc = Kc = 0
    Ma = T * kg
    for l in range(1, n + 1):
        m, e, x = bin_counts(_group(s, l - 1, kg), _group(t, l - 1, kg))
        Mc += m
        Kc += effective_bins(kg, e, x, rule)
        if l == n:
            return (ACCEPT if Kc > 0 and Mc >= T * Kc else REJECT), l, Mc
        Mra = (T * (Kc + (n - l) * kg) - Mc) / (n - l)
        if Mra < Ma:
            if bt.lower(Mra) <= eps:
                return ACCEPT, l, Mc
        else:
            if bt.upper(Mra) <= eps:
                return REJECT, l, Mc
    raise AssertionError("unreachable")


def hoph_compare(s, t, kg, z, T, eps, rule="both", weighting="space", ab=None):
    """(a:b)HOPH comparison (Algorithm 2, Sec. 4.1) of two sketches laid out
    in groups of k' bins with space sizes z[0..G-1].  Returns
    (decision, groups compared, matched bins).

    weighting='space': after l groups, with D_l the compared groups that have
    a non-empty bin, S = sum_{j in D_l} z_j M_j / K_j, Z_done = sum z_j over
    D_l, Z_rem = sum of the sizes not yet compared:
        P_r = (T*(Z_done + Z_rem) - S) / Z_rem.
    weighting='literal': Algorithm 2's recursion P <- (P - (M_l/k') r^l)/r^l
    from P = T, r = a/(a+b) (``ab`` = (a, b)).
    Then: P_r < T and P(X < P_r k') <= eps -> similar; P_r >= T and
    P(X >= P_r k') <= eps -> not similar; else next group.  After all G
    groups: similar iff Z_done > 0 and S >= T Z_done (Lemma 3's estimator,
    space-weighted, >= T)."""
    T = Fraction(T)
    eps = Fraction(eps)
    G = len(z)
    bt = BinomialTails(kg, T)
    S = Fraction(0)
    Zd = 0
    Mc = 0
    P = T
    if weighting == "literal":
        a, b = ab
        r = Fraction(a, a + b)
    for l in range(1, G + 1):
        m, e, x = bin_counts(_group(s, l - 1, kg), _group(t, l - 1, kg))
        K = effective_bins(kg, e, x, rule)
        Mc += m
        if K > 0:
            S += Fraction(z[l - 1] * m, K)
            Zd += z[l - 1]
        if l == G:
            return (ACCEPT if Zd > 0 and S >= T * Zd else REJECT), l, Mc
        if weighting == "space":
            Zrem = sum(z[l:])
            Pr = (T * (Zd + Zrem) - S) / Zrem
        elif weighting == "literal":
            Pr = (P - Fraction(m, kg) * r ** l) / r ** l
            P = Pr
        else:
            raise ValueError(weighting)
        if Pr < T:
            if bt.lower(Pr * kg) <= eps:
                return ACCEPT, l, Mc
        else:
            if bt.upper(Pr * kg) <= eps:
                return REJECT, l, Mc
    raise AssertionError("unreachable")


def oph_full_compare(s, t, T, rule="both"):
    """Plain OPH (Eq. 6): R = N_mb / (k - N_eb) over all k bins, similar iff
    k - N_eb > 0 and R >= T.  Returns (decision, 1, matched bins)."""
    T = Fraction(T)
    m, e, x = bin_counts(s, t)
    K = effective_bins(len(s), e, x, rule)
    return (ACCEPT if K > 0 and m >= T * K else REJECT), 1, m


def minwise_compare(s, t, T):
    """MinWise: the fraction of the k minima that agree, similar iff >= T."""
    T = Fraction(T)
    m = sum(1 for u, v in zip(s, t) if u != EMPTY and u == v)
    return (ACCEPT if m >= T * len(s) else REJECT), 1, m


def oph_estimate(s, t, rule="both"):
    """R_mb = N_mb / (k - N_eb) (Eq. 6) as an exact Fraction (None if k = N_eb)."""
    m, e, x = bin_counts(s, t)
    K = effective_bins(len(s), e, x, rule)
    return Fraction(m, K) if K else None


def hoph_estimate(s, t, kg, z, rule="both"):
    """Lemma 3's estimator with space weights: sum z_j M_j/K_j / sum z_j over
    groups with K_j > 0 (None if no group has a non-empty bin)."""
    S = Fraction(0)
    Zd = 0
    for g in range(len(z)):
        m, e, x = bin_counts(_group(s, g, kg), _group(t, g, kg))
        K = effective_bins(kg, e, x, rule)
        if K:
            S += Fraction(z[g] * m, K)
            Zd += z[g]
    return S / Zd if Zd else None


# ---------------------------------------------------------------------------
# Ground truth and metrics (Sec. 3.1, Sec. 5)
# ---------------------------------------------------------------------------

def exact_jaccard(A, B):
    """|A n B| / |A u B| on the distinct elements (0 for two empty sets)."""
    A = set(A)
    B = set(B)
    u = len(A | B)
    return Fraction(len(A & B), u) if u else Fraction(0)


def precision_recall(retrieved, relevant):
    """Precision and recall as defined in Sec. 5 ("performance metric")."""
    retrieved = set(retrieved)
    relevant = set(relevant)
    hit = len(retrieved & relevant)
    precision = Fraction(hit, len(retrieved)) if retrieved else Fraction(1)
    recall = Fraction(hit, len(relevant)) if relevant else Fraction(1)
    return precision, recall
