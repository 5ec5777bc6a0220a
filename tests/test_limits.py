"""The small-probability limits U and L of Definition 1 (X ~ Bin(k', T);
the two tails of Eq. 10-11 that Table 2 prints), compared with the exact
Fraction tails of the oracle, including tolerances eps set exactly on a
tail's double value and one ulp to either side, where rounded arithmetic
and exact arithmetic part ways.  The library's host routine and the C
oracle's tail test are checked without a GPU; every plan's limits are
checked on the GPU."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import hoph_ref as hr
from oracle import oracle_c as oc
from paper_1805_11254_gb300 import build_lib, hoph

KGS = (16, 32, 64, 100, 128)
THRS = ((3, 5), (7, 10), (4999, 7001), (1, 3))


def _eps_grid(kg, thr):
    """0, 1, a few round tolerances, and every tail's nearest double with its
    two neighbours (the tails that fit a double's range)."""
    bt = hr.BinomialTails(kg, Fraction(*thr))
    out = {0.0, 1.0, 1e-4, 1e-3, 1e-12, 0.5, 2.0}
    for tails in (bt.up, bt.low):
        for v in tails:
            f = float(v)
            if 0.0 < f < 1.0:
                out.update((f, math.nextafter(f, 0.0), math.nextafter(f, 2.0)))
    return sorted(out)


def _exact(kg, thr, eps):
    return hr.small_probability_limits(kg, Fraction(*thr), eps)


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return hoph.load()


@pytest.mark.parametrize("kg", KGS)
@pytest.mark.parametrize("thr", THRS)
def test_library_limits_equal_the_exact_tails(lib, kg, thr):
    for eps in _eps_grid(kg, thr):
        got = hoph.hoph_small_probability_limits(kg, thr[0], thr[1], eps)
        assert got == _exact(kg, thr, eps), (kg, thr, eps)


def test_limits_at_an_exact_dyadic_tail():
    """T = 1/2: every tail is a dyadic rational, so eps can equal a tail
    exactly; the comparison is <= (Definition 1)."""
    hoph.load()
    for kg in (8, 31, 64):
        bt = hr.BinomialTails(kg, Fraction(1, 2))
        for j in range(kg + 2):
            for v in (bt.up[j], bt.low[j]):
                f = float(v)
                if Fraction(f) != v or not 0 < f < 1:
                    continue
                for eps in (f, math.nextafter(f, 0.0), math.nextafter(f, 2.0)):
                    assert (hoph.hoph_small_probability_limits(kg, 1, 2, eps)
                            == hr.small_probability_limits(kg, Fraction(1, 2), eps)), (kg, j, eps)


def test_limits_known_values_and_edges():
    hoph.load()
    f = hoph.hoph_small_probability_limits
    assert f(100, 3, 5, 1e-4) == (79, 42)                 # Example 2's k' and T
    assert f(64, 7, 10, 1e-4) == (58, 31)
    assert f(64, 7, 10, 0.0) == (65, 0)                   # eps = 0: only impossibility
    assert f(64, 7, 10, 1.0) == (0, 65)                   # eps >= 1: every tail
    assert f(64, 10, 10, 1e-4) == (65, 64)                # T = 1: X = k'
    assert f(64, 14, 20, 1e-4) == f(64, 7, 10, 1e-4)      # T in lowest terms
    with pytest.raises(hoph.HophError):
        f(0, 7, 10, 1e-4)
    with pytest.raises(hoph.HophError):
        f(64, 11, 10, 1e-4)
    with pytest.raises(hoph.HophError):
        f(64, 7, 10, -1.0)
    with pytest.raises(hoph.HophError):
        f(64, 7, 10, float("nan"))


def test_limits_large_k_prime_stay_exact_and_fast():
    """Where long double would underflow (0.5^4096 is fine, 0.3^20000 is
    not): a large k' is still decided exactly, and quickly."""
    import time
    hoph.load()
    t0 = time.perf_counter()
    U, L = hoph.hoph_small_probability_limits(20000, 7, 10, 1e-4)
    assert time.perf_counter() - t0 < 10
    mean, sd = 14000, math.sqrt(20000 * 0.21)
    assert mean < U < mean + 6 * sd and mean - 6 * sd < L < mean
    # a tail far below the smallest long double still compares exactly
    U0, L0 = hoph.hoph_small_probability_limits(20000, 7, 10, 5e-324)
    assert U0 > U and L0 < L


@pytest.mark.parametrize("kg", KGS)
@pytest.mark.parametrize("thr", THRS)
def test_c_oracle_tail_tests_equal_the_exact_tails(kg, thr):
    oc.build()
    for eps in _eps_grid(kg, thr):
        assert oc.limits(kg, thr[0], thr[1], eps) == _exact(kg, thr, eps), (kg, thr, eps)


@pytest.mark.gpu
def test_plan_limits_equal_the_exact_tails():
    """Every plan's U and L (hoph_plan_info) equal the exact limits."""
    for kg in KGS:
        for thr in THRS:
            for eps in _eps_grid(kg, thr)[::3] + [0.0, 1e-4, 1.0]:
                with hoph.Plan(1 << 12, kg, kg, seed=1, thr=thr, epsilon=eps) as p:
                    got = (p.info.upper_limit, p.info.lower_limit)
                assert got == _exact(kg, thr, eps), (kg, thr, eps)
