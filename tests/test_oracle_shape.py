"""Oracle pins: splitting-tree shape (Section 2.2, "Splitting Trees").

The lower aggregation fanouts are max(2, ceil(0.35 l + 0.55)) and
max(2, ceil(0.21 l + 0.9)); the upper levels use fanout 2.  Exact rational
arithmetic below gives the ceilings without floating-point doubt.
"""
import os
from fractions import Fraction
from math import ceil

import pytest


def paper_fanouts(leaf):
    f1 = max(2, ceil(Fraction(35, 100) * leaf + Fraction(55, 100)))
    f2 = max(2, ceil(Fraction(21, 100) * leaf + Fraction(90, 100)))
    return f1, f2


@pytest.mark.parametrize("leaf", range(2, 25))
def test_fanouts_follow_the_paper_formula(orc, leaf):
    assert orc.fanouts(leaf) == paper_fanouts(leaf)


def test_fanouts_of_the_benchmark_leaf_sizes(orc):
    assert orc.fanouts(8) == (4, 3)
    assert orc.fanouts(12) == (5, 4)
    assert orc.fanouts(16) == (7, 5)


@pytest.mark.parametrize("leaf", [2, 3, 5, 7, 8, 10, 12, 16, 24])
def test_parts_partition_every_node(orc, leaf):
    f1, f2 = orc.fanouts(leaf)
    lower1, lower2 = f1 * leaf, f1 * f2 * leaf
    for m in range(0, 4097, 1 if leaf in (8, 16) else 7):
        p = orc.parts(leaf, m)
        if m <= leaf:
            assert p == []
            continue
        assert sum(p) == m and all(x >= 1 for x in p)
        if m <= lower1:
            assert len(p) <= f1 and all(x == leaf for x in p[:-1]) and p[-1] <= leaf
        elif m <= lower2:
            assert len(p) <= f2 and all(x == lower1 for x in p[:-1]) and p[-1] <= lower1
        else:
            assert len(p) == 2
            left, right = p
            assert left % lower2 == 0 and left >= m // 2 and right >= 1
            # the SMALLEST such multiple (reading of the fanout-2 left size):
            # one unit less would fall below floor(m/2)
            assert left - lower2 < m // 2


@pytest.mark.parametrize("leaf", [4, 8, 12, 16])
def test_leaves_cover_every_key_once(orc, leaf):
    """Leaves (nodes of at most l keys) tile the bucket: sizes sum to m and
    all are full except at most one per lower-1 node."""
    def leaves(m):
        if m <= leaf:
            return [m]
        out = []
        for p in orc.parts(leaf, m):
            out += leaves(p)
        return out

    for m in (1, 2, leaf, leaf + 1, 100, 999, 2000, 2313, 4096):
        ls = leaves(m)
        assert sum(ls) == m
        assert all(1 <= x <= leaf for x in ls)


def test_node_counts(orc):
    assert orc.count_nodes(16, 0) == 0
    assert orc.count_nodes(16, 1) == 0
    assert orc.count_nodes(16, 2) == 1
    assert orc.count_nodes(16, 16) == 1
    assert orc.count_nodes(16, 112) == 8          # root + 7 leaves
    assert orc.count_nodes(16, 560) == 1 + 5 * 8  # root + 5 lower-1 subtrees
    assert orc.count_nodes(16, 17) == 2           # root + leaf of 16 (the leftover key is not stored)
    assert orc.count_nodes(16, 18) == 3
    # a fanout-2 root over two lower-2 nodes
    assert orc.count_nodes(16, 1120) == 1 + 2 * 41


def test_salts_distinct(orc):
    salts = [orc.salt(l) for l in range(40)]
    assert len(set(salts)) == 40


def test_salts_are_the_published_splitmix64_outputs(orc):
    """salt(L) = mix64((L + 1) G) is output L of SplitMix64 started from state
    0 (Steele, Lea and Flood, OOPSLA 2014), whose first outputs are published.
    An off-by-one in the level index (mix64(L G)) or a wrong increment fails."""
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", "splitmix64_seed0.txt")) as f:
        golden = [int(line, 16) for line in f if line.strip() and not line.startswith("#")]
    assert len(golden) == 4
    assert [orc.salt(level) for level in range(4)] == golden
