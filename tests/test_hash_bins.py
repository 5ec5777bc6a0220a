"""The hashed-psi sketch finds a value's bin inside an equal-width region
(one region per group of an (a:b) layout, the whole space for equal bins) as
the high 64-bit word of o * magic, magic = floor(2^64 nb / z) + 1, instead of
dividing: o nb / z exceeds floor(o nb / z) by at most 1 - 1/z while
o * magic / 2^64 exceeds o nb / z by less than o / 2^64 < 2^-32 <= 1/z.
These checks hold the identity against exact integer division on the
layouts the sketch path serves (D = 2^32), at every bin's lower bound, one
below and one above it, and at random offsets, and against the bins of the
oracle's layout."""
import numpy as np
import pytest

from oracle import hoph_ref as hr


def _magic(nb, z):
    return ((nb << 64) // z) + 1 if nb < z else 0


def _bin(o, nb, z, m):
    # the kernel's two 32-bit products: o * (m >> 32) + hi32(o * (m & 0xFFFFFFFF)), >> 32
    if m == 0:
        return o
    t = (o * (m & 0xFFFFFFFF)) >> 32
    return (o * (m >> 32) + t) >> 32


@pytest.mark.parametrize("k,kg,a,b", [(512, 128, 2, 1), (512, 128, 1, 2), (256, 64, 1, 1),
                                      (128, 128, 0, 0), (1024, 256, 3, 1)])
def test_magic_bin_equals_the_division_at_every_boundary(k, kg, a, b):
    D = 1 << 32
    lo, _ = hr.layout(D, k, kg, a, b)
    lo = [int(x) for x in lo]
    equal = a == 0 and b == 0
    regions = [(0, k)] if equal else [(g * kg, kg) for g in range(k // kg)]
    rng = np.random.default_rng(k + kg + a)
    for first, nb in regions:
        start, z = lo[first], lo[first + nb] - lo[first]
        m = _magic(nb, z)
        assert m < 1 << 64
        offs = set()
        for j in range(nb):
            o = lo[first + j] - start
            offs.update((o, o + 1, max(o - 1, 0)))
        offs.update(int(x) for x in rng.integers(0, z, 2000))
        offs.add(z - 1)
        for o in sorted(x for x in offs if x < z):
            q = _bin(o, nb, z, m)
            assert q == o * nb // z, (first, o)
            # ... and that is the bin of the oracle's layout holding the value
            assert lo[first + q] <= start + o < lo[first + q + 1]


def test_bins_of_one_value_take_the_offset():
    assert _magic(5, 5) == 0
    assert [_bin(o, 5, 5, 0) for o in range(5)] == [0, 1, 2, 3, 4]
