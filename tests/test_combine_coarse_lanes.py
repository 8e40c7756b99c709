"""The combination kernel's coarse phase, restated in plain Python (CPU
only): the terms of the coarse Horner levels, pairs (l, x) with l from the
first level L0 to ltop = min(n, 5) and x < 2^l, are numbered
p = 2^l - 2^L0 + x and computed two per lane (p = lane and lane + 32).  Lane
x of level l then takes pair p = 2^l - 2^L0 + x by a shuffle from lane
p mod 32, slot p div 32.  Checked for every level range the kernel meets:
each pair is computed exactly once, with l and x recovered from p, and every
lane reads the pair it needs."""
import pytest


def pairs_by_lane(L0, ltop):
    p0 = 1 << L0
    npairs = (2 << ltop) - p0
    assert npairs <= 64
    got = {}
    for lane in range(32):
        for slot in range(2):
            p = lane + 32 * slot
            if p < npairs:
                l = (p + p0).bit_length() - 1  # 31 - clz(p + p0)
                x = p + p0 - (1 << l)
                got[(lane, slot)] = (l, x)
    return got


@pytest.mark.parametrize("n", range(2, 13))
@pytest.mark.parametrize("lmin", range(0, 7))
@pytest.mark.parametrize("cell", [False, True])
def test_coarse_pairs(n, lmin, cell):
    L0 = min(lmin + 1 if cell else lmin, min(n, 5))
    ltop = min(n, 5)
    got = pairs_by_lane(L0, ltop)
    want = {(l, x) for l in range(L0, ltop + 1) for x in range(1 << l)}
    assert sorted(got.values()) == sorted(want)  # every pair once
    for l in range(L0, ltop + 1):
        for lane in range(1 << l):
            p = (1 << l) - (1 << L0) + lane
            assert got[(p & 31, p >> 5)] == (l, lane)
