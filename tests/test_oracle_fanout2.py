"""Oracle pins: the fanout-2 splitting tree (Appendix C).

With ShockHash leaves the paper sets the fanout to 2 for the whole tree, so
larger leaves can be used.  Every inner node of m keys then splits in two,
the left part the smallest multiple of l that is at least floor(m/2).  Pins:

* shape: the parts of every node size partition it, the left part is a
  multiple of l and at least floor(m/2), leaves cover every key once, and the
  node count satisfies nodes(m) = 1 + nodes(left) + nodes(right);
* every split and leaf is minimal by brute force on tiny inputs, for all
  three leaf methods (ShockHash leaves through the ShockHash checker);
* queries are bijections; the Golomb-Rice stream decodes back to the values;
* the split trial counts match the binomial success probability
  C(m, left) (left/m)^left (right/m)^right.
"""
import math

import numpy as np
import pytest

from helpers import NaiveChecker, group_by_bucket
from paper_2212_09562_b300 import workloads as W
from test_oracle_encoding import bits_of
from test_oracle_shockhash import ShockChecker

F2 = 1  # oracle tree code: fanout 2 everywhere


@pytest.mark.parametrize("leaf", [2, 3, 5, 8, 12, 16, 24])
def test_fanout2_shape(orc, leaf):
    assert orc.fanouts(leaf, F2) == (1, 1)
    for m in range(2, 4097):
        p = orc.parts(leaf, m, F2)
        if m <= leaf:
            assert p == [] and orc.count_nodes(leaf, m, F2) == 1
            continue
        assert len(p) == 2 and sum(p) == m
        assert p[0] % leaf == 0 and p[0] >= m // 2 and p[0] - leaf < m // 2
        assert p[1] >= 1
        assert orc.count_nodes(leaf, m, F2) == 1 + orc.count_nodes(leaf, p[0], F2) + \
            orc.count_nodes(leaf, p[1], F2)


def _leaf_sizes(orc, leaf, m):
    if m <= leaf:
        return [m]
    return [s for q in orc.parts(leaf, m, F2) for s in _leaf_sizes(orc, leaf, q)]


@pytest.mark.parametrize("leaf", [3, 8, 24])
def test_fanout2_leaves_cover_every_key_once(orc, leaf):
    for m in (1, 2, leaf, leaf + 1, 3 * leaf + 1, 1000, 4096):
        sizes = _leaf_sizes(orc, leaf, m)
        assert sum(sizes) == m and all(1 <= s <= leaf for s in sizes)


@pytest.mark.parametrize("leaf,bucket,rotation,kb,n", [
    (4, 30, False, 8, 200), (4, 30, True, 8, 200), (5, 60, True, 16, 300), (3, 50, False, 8, 150),
    (2, 20, True, 8, 80),
])
def test_fanout2_nodes_are_minimal_by_brute_force(orc, leaf, bucket, rotation, kb, n):
    keys = W.random_keys(n, kb, 700 + leaf)
    h = orc.build_mphf(keys, leaf, bucket, rotation, tree=F2)
    hi, lo, groups = group_by_bucket(orc, keys, h.nb)
    chk = NaiveChecker(orc, leaf, rotation, tree=F2)
    checked = 0
    for b in range(h.nb):
        idx = groups.get(b, [])
        vals = h.values[int(h.node_off[b]):int(h.node_off[b + 1])]
        checked += chk.check_bucket(lo[idx], hi[idx], vals)
    assert checked == h.n_nodes and checked > 10


class _ShockTree(NaiveChecker):
    """The naive tree walk with ShockHash leaves checked by brute force."""

    def __init__(self, orc, leaf):
        super().__init__(orc, leaf, False, tree=F2)
        self.sh = ShockChecker(orc)
        self.mask = (1 << orc.SH_SEED_BITS) - 1
        self.bits = orc.SH_SEED_BITS

    def _node(self, lo, hi, m, depth, it, max_brute):
        if 2 <= m <= self.leaf:
            x = int(next(it))
            s, z = x & self.mask, x >> self.bits
            lo = [int(v) for v in lo]
            got = self.sh.accepts(lo, s, m)
            assert got is not None and z in got[3]
            assert all(self.sh.accepts(lo, t, m) is None for t in range(s))
            return 1
        return super()._node(lo, hi, m, depth, it, max_brute)


@pytest.mark.parametrize("leaf,bucket,n", [(4, 40, 300), (6, 100, 400), (8, 50, 300)])
def test_fanout2_shockhash_nodes_are_minimal_by_brute_force(orc, leaf, bucket, n):
    keys = W.distinct_u64(n, 720 + leaf)
    h = orc.build_mphf(keys, leaf, bucket, orc.SHOCKHASH, tree=F2)
    hi, lo, groups = group_by_bucket(orc, keys, h.nb)
    chk = _ShockTree(orc, leaf)
    checked = 0
    for b in range(h.nb):
        idx = groups.get(b, [])
        vals = h.values[int(h.node_off[b]):int(h.node_off[b + 1])]
        checked += chk.check_bucket(lo[idx], hi[idx], vals)
    assert checked == h.n_nodes and checked > 10


@pytest.mark.parametrize("leaf,bucket,rotation,kb,n", [
    (8, 100, False, 8, 20000), (8, 2000, True, 16, 20000), (12, 1000, True, 8, 8000),
    (16, 2000, 2, 8, 30000), (24, 2000, 2, 16, 20000), (20, 3000, 2, 8, 9000), (2, 5, 2, 8, 700),
    (24, 7, 2, 8, 500), (8, 100, 2, 8, 1),
])
def test_fanout2_query_is_a_bijection(orc, leaf, bucket, rotation, kb, n):
    keys = W.random_keys(n, kb, 740 + leaf)
    h = orc.build_mphf(keys, leaf, bucket, rotation, threads=4, tree=F2)
    q = h.query(keys)
    assert np.array_equal(np.sort(q), np.arange(n, dtype=np.uint64))


def _preorder(orc, leaf, m):
    if m <= 1:
        return []
    out = [m]
    if m > leaf:
        for p in orc.parts(leaf, m, F2):
            out += _preorder(orc, leaf, p)
    return out


@pytest.mark.parametrize("leaf,rotation", [(16, 2), (8, True)])
def test_fanout2_golomb_rice_round_trip(orc, leaf, rotation):
    keys = W.distinct_u64(8000, 760 + leaf)
    h = orc.build_mphf(keys, leaf, 1000, rotation, tree=F2)
    tau = orc.tau_table(leaf, rotation, tree=F2)
    shock = int(rotation) == orc.SHOCKHASH
    mask = (1 << orc.SH_SEED_BITS) - 1
    for b in range(h.nb):
        m = int(h.cum_keys[b + 1] - h.cum_keys[b])
        sizes = _preorder(orc, leaf, m)
        vals = h.values[int(h.node_off[b]):int(h.node_off[b + 1])]
        pos = int(h.bit_pos[b])
        fixed, zs = [], []
        for s in sizes:
            fixed.append(bits_of(h.gr, pos, int(tau[s])))
            pos += int(tau[s])
            z = 0
            if shock and s <= leaf:
                z = bits_of(h.gr, pos, s)
                pos += s
            zs.append(z)
        for s, f, z, v in zip(sizes, fixed, zs, vals):
            zeros = 0
            while not (int(h.gr[pos >> 6]) >> (pos & 63)) & 1:
                zeros += 1
                pos += 1
            pos += 1
            seed = (zeros << int(tau[s])) | f
            if shock and s <= leaf:
                assert seed == int(v) & mask and z == int(v) >> orc.SH_SEED_BITS
            else:
                assert seed == int(v)
        assert pos == int(h.bit_pos[b + 1])


@pytest.mark.parametrize("leaf,m,count", [(8, 16, 3000), (8, 40, 2000), (24, 100, 1500)])
def test_fanout2_split_trials_match_the_binomial(orc, leaf, m, count):
    left, right = orc.parts(leaf, m, F2)
    p = math.comb(m, left) * (left / m) ** left * (right / m) ** right
    rng = np.random.default_rng(780 + m)
    t = []
    for _ in range(count):
        lo = rng.integers(0, 2**63, m, dtype=np.int64).astype(np.uint64)
        rc, x, trials, evals = orc.node_search(leaf, False, lo, depth=1, tree=F2)
        assert rc == 0 and evals == trials * m
        t.append(trials)
    t = np.asarray(t, float)
    assert abs(t.mean() - 1 / p) < 4 * t.std(ddof=1) / math.sqrt(count)
    assert orc.split_success(leaf, m, F2) == pytest.approx(p, rel=1e-9)
