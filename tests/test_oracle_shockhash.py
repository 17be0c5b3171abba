"""Oracle pins: ShockHash leaves (Appendix C).

A ShockHash leaf stores a seed s under which the two cells of every key
admit a bijection, plus one retrieved bit per key that says which cell the
key takes.  What pins the oracle, each by a route of its own:

* The success probability of a trial (every component of the cuckoo graph
  has as many keys as cells): exhaustive enumeration of all cell pairs for
  m <= 4, the values 7/8 and 58/81 derived by hand for m = 2, 3, and the
  paper's statement that p behaves like 2^(-0.44 m) for large m.
* The solvability of the retrieval system: exhaustive enumeration of all
  GF(2) matrices and right-hand sides for m <= 3.
* Minimality by brute force on tiny leaves: for the stored seed, the stored
  retrieval vector selects a bijection, the selected bits are the canonical
  choice (found by enumerating every bijection and locating the cycle edges
  as the non-bridges), and the vector is the one with zeros at the columns
  that depend on earlier columns (enumeration over all 2^m vectors); every
  smaller seed admits no bijection or has no solution for its canonical bits
  (enumeration again).
* End to end: the query is a bijection onto [0, n); the Golomb-Rice stream
  decodes back to the stored seeds and retrieval vectors; the mean number of
  trials per leaf matches 1 / (P(bijection) P(solvable)).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from helpers import M64
from paper_2212_09562_b300 import workloads as W
from test_oracle_encoding import bits_of, preorder_sizes


def _orientable_brute(c0, c1, m):
    """Some choice of one cell per key is a bijection (try all 2^m choices)."""
    for bits in itertools.product((0, 1), repeat=len(c0)):
        if len({(c1[i] if b else c0[i]) for i, b in enumerate(bits)}) == m:
            return True
    return False


def test_bijection_probability_by_enumeration(orc):
    assert orc.shockhash_orient_prob(1) == 1.0
    assert orc.shockhash_orient_prob(2) == pytest.approx(7 / 8, abs=1e-15)
    assert orc.shockhash_orient_prob(3) == pytest.approx(58 / 81, abs=1e-15)
    for m in (2, 3, 4):
        cells = np.array(list(itertools.product(range(m), repeat=2 * m)), dtype=np.int8)
        c0, c1 = cells[:, 0::2], cells[:, 1::2]  # (lists, m)
        ok = np.zeros(len(cells), bool)
        for bits in itertools.product((0, 1), repeat=m):
            chosen = np.where(np.array(bits, bool)[None, :], c1, c0)
            s = np.sort(chosen, axis=1)
            ok |= np.all(s == np.arange(m)[None, :], axis=1)
        exact = Fraction(int(ok.sum()), m ** (2 * m))
        assert orc.shockhash_orient_prob(m) == pytest.approx(float(exact), rel=1e-13)


def test_bijection_probability_tends_to_the_papers_rate(orc):
    """Appendix C: p -> 2^(-0.44 m).  The exponent per key falls monotonically
    towards that rate (about log2(e/2) = 0.4427) and stays above it."""
    rates = [-math.log2(orc.shockhash_orient_prob(m)) / m for m in range(4, 25)]
    assert all(b > a for a, b in zip(rates, rates[1:]))
    assert 0.37 < rates[-1] < 0.4427


def test_retrieval_solvable_probability_by_enumeration(orc):
    for m in (1, 2, 3):
        rows = list(itertools.product(range(1 << m), repeat=m))
        good = total = 0
        for rhs in range(1, 1 << m):
            for r in rows:
                total += 1
                good += any(all(((bin(r[i] & z).count("1") & 1) == ((rhs >> i) & 1))
                                for i in range(m)) for z in range(1 << m))
        assert orc.retrieval_solvable_prob(m) == pytest.approx(good / total, rel=1e-13)
    # a large random system: about 0.61 (the rank deficiency of random GF(2) matrices)
    assert orc.retrieval_solvable_prob(24) == pytest.approx(0.6103, abs=1e-4)


class ShockChecker:
    """Brute-force restatement of a ShockHash leaf from the definitions."""

    def __init__(self, orc):
        self.orc = orc
        self.s0 = orc.salt(0)
        self.sr = orc.salt(orc.SH_RETRIEVAL_LEVEL)

    def cells(self, lo, s, m):
        c0, c1 = [], []
        for x in lo:
            h = self.orc.mix64((int(x) + self.s0 + s) & M64)
            c0.append((h & 0xFFFFFFFF) % m)
            c1.append((h >> 32) % m)
        return c0, c1

    def rows(self, lo, s, m):
        return [self.orc.mix64((int(x) + self.sr + s) & M64) & ((1 << m) - 1) for x in lo]

    @staticmethod
    def _connected(m, edges):
        parent = list(range(m))

        def find(a):
            while parent[a] != a:
                a = parent[a]
            return a

        for u, v in edges:
            parent[find(u)] = find(v)
        return [find(v) for v in range(m)]

    def canonical_bits(self, lo, c0, c1, m):
        """Among all bijective choices, the one where on every cycle the key
        with the smallest lo word takes its first cell; the cycle keys are the
        edges whose removal keeps their component connected."""
        edges = list(zip(c0, c1))
        comp = self._connected(m, edges)
        on_cycle = []
        for i in range(len(edges)):
            rest = self._connected(m, edges[:i] + edges[i + 1:])
            u, v = edges[i]
            on_cycle.append(rest[u] == rest[v])
        lead = {}
        for i in range(len(edges)):
            if on_cycle[i]:
                c = comp[c0[i]]
                if c not in lead or lo[i] < lo[lead[c]]:
                    lead[c] = i
        found = []
        for bits in itertools.product((0, 1), repeat=len(edges)):
            if len({(c1[i] if b else c0[i]) for i, b in enumerate(bits)}) != m:
                continue
            if all(bits[i] == 0 for i in lead.values()):
                found.append(bits)
        assert len(found) == 1
        return found[0]

    @staticmethod
    def solutions(rows, bits, m):
        return [z for z in range(1 << m)
                if all((bin(r & z).count("1") & 1) == b for r, b in zip(rows, bits))]

    @staticmethod
    def dependent_columns(rows, m):
        """Columns in the span of the columns before them."""
        cols = [sum(((r >> j) & 1) << i for i, r in enumerate(rows)) for j in range(m)]
        dep = []
        for j in range(m):
            span = {0}
            for c in cols[:j]:
                span |= {x ^ c for x in span}
            dep.append(cols[j] in span)
        return dep

    def accepts(self, lo, s, m):
        c0, c1 = self.cells(lo, s, m)
        if not _orientable_brute(c0, c1, m):
            return None
        bits = self.canonical_bits(lo, c0, c1, m)
        sols = self.solutions(self.rows(lo, s, m), bits, m)
        return (c0, c1, bits, sols) if sols else None


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7, 8])
def test_shockhash_leaf_is_minimal_by_brute_force(orc, m):
    rng = np.random.default_rng(500 + m)
    chk = ShockChecker(orc)
    for _ in range(12 if m <= 6 else 5):
        lo = [int(v) for v in rng.integers(0, 2**63, m, dtype=np.int64)]
        rc, x, trials, evals = orc.node_search(m, orc.SHOCKHASH, np.array(lo, np.uint64))
        assert rc == 0
        s, z = x & ((1 << orc.SH_SEED_BITS) - 1), x >> orc.SH_SEED_BITS
        assert trials == s + 1 and evals == m * trials
        got = chk.accepts(lo, s, m)
        assert got is not None
        c0, c1, bits, sols = got
        assert z in sols
        dep = chk.dependent_columns(chk.rows(lo, s, m), m)
        canon = [v for v in sols if all(not ((v >> j) & 1) for j in range(m) if dep[j])]
        assert canon == [z]
        # the retrieved bits select the canonical bijection
        rows = chk.rows(lo, s, m)
        picked = [c1[i] if (bin(rows[i] & z).count("1") & 1) else c0[i] for i in range(m)]
        assert sorted(picked) == list(range(m))
        assert all(chk.accepts(lo, t, m) is None for t in range(s))


@pytest.mark.parametrize("m,count,seed", [(8, 3000, 61), (16, 6000, 901), (24, 600, 85)])
def test_shockhash_trials_match_the_success_probability(orc, m, count, seed):
    rng = np.random.default_rng(seed)
    t = []
    for _ in range(count):
        lo = rng.integers(0, 2**63, m, dtype=np.int64).astype(np.uint64)
        rc, x, trials, evals = orc.node_search(m, orc.SHOCKHASH, lo)
        assert rc == 0
        t.append(trials)
    t = np.asarray(t, float)
    expected = 1.0 / (orc.shockhash_orient_prob(m) * orc.retrieval_solvable_prob(m))
    # the all-zero bit vector is always solvable, so the true mean is a little lower
    assert abs(t.mean() - expected) < 4 * t.std(ddof=1) / math.sqrt(count) + 0.03 * expected


@pytest.mark.parametrize("leaf,bucket,kb,n", [(8, 100, 8, 20000), (4, 30, 16, 3000), (12, 500, 8, 8000),
                                              (2, 5, 8, 500), (16, 2000, 16, 3000), (24, 100, 8, 1500),
                                              (8, 100, 8, 9)])
def test_shockhash_query_is_a_bijection(orc, leaf, bucket, kb, n):
    keys = W.random_keys(n, kb, 90 + leaf)
    h = orc.build_mphf(keys, leaf, bucket, orc.SHOCKHASH, threads=4)
    q = h.query(keys)
    assert np.array_equal(np.sort(q), np.arange(n, dtype=np.uint64))


@pytest.mark.parametrize("leaf,bucket,n", [(8, 100, 6000), (5, 23, 2000), (12, 1000, 4000)])
def test_shockhash_golomb_rice_round_trip(orc, leaf, bucket, n):
    """Fixed part of a ShockHash leaf: tau bits of the seed, then its m
    retrieval bits; unary part: the seed's high bits."""
    keys = W.distinct_u64(n, 95 + leaf)
    h = orc.build_mphf(keys, leaf, bucket, orc.SHOCKHASH)
    tau = orc.tau_table(leaf, orc.SHOCKHASH)
    mask = (1 << orc.SH_SEED_BITS) - 1
    for b in range(h.nb):
        m = int(h.cum_keys[b + 1] - h.cum_keys[b])
        sizes = preorder_sizes(orc, leaf, m)
        vals = h.values[int(h.node_off[b]):int(h.node_off[b + 1])]
        pos = int(h.bit_pos[b])
        fixed, zs = [], []
        for s in sizes:
            fixed.append(bits_of(h.gr, pos, int(tau[s])))
            pos += int(tau[s])
            if s <= leaf:
                zs.append(bits_of(h.gr, pos, s))
                pos += s
            else:
                zs.append(0)
        for s, f, zv, v in zip(sizes, fixed, zs, vals):
            zeros = 0
            while not (int(h.gr[pos >> 6]) >> (pos & 63)) & 1:
                zeros += 1
                pos += 1
            pos += 1
            seed = (zeros << int(tau[s])) | f
            if s <= leaf:
                assert seed == int(v) & mask and zv == int(v) >> orc.SH_SEED_BITS
            else:
                assert seed == int(v)
        assert pos == int(h.bit_pos[b + 1])
    assert int(h.bit_pos[-1]) == h.gr_bits


def test_shockhash_search_cap(orc):
    keys = W.distinct_u64(2000, 97)
    with pytest.raises(orc.OracleError) as e:
        orc.build_mphf(keys, 8, 100, orc.SHOCKHASH, max_value=2)
    assert e.value.code == orc.ESEARCH_LIMIT
    with pytest.raises(ValueError):
        orc.build_mphf(keys, 8, 100, 3)  # no such leaf method
    import ctypes
    h = ctypes.c_void_p()
    rc = orc.lib().orc_build(keys.ctypes.data, len(keys), 8, 8, 100, 3, orc.DEFAULT_MAX_VALUE, 1,
                             ctypes.byref(h))
    assert rc == orc.EINVAL and not h.value
