"""Shared test helpers: golden fixtures and a deliberately naive checker.

The checker re-derives every node of a built function on tiny inputs and
verifies, by brute force, that the stored value works and that every smaller
value fails (the method stores the smallest working value; Section 5.1,
"Bijections", on trying all rotations).  Rotation leaves are checked with the
query-time rule of Section 4: keys of B move by +r mod m.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
M64 = (1 << 64) - 1


def golden_pairs(name: str) -> list[tuple[float, float]]:
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b = line.split()
            out.append((float(a), float(b)))
    return out


def golden_hex(name: str) -> list[int]:
    with open(os.path.join(GOLDEN, name)) as f:
        return [int(l, 16) for l in f if l.strip() and not l.startswith("#")]


class NaiveChecker:
    """Walks each bucket's tree from the stored values and checks every node."""

    def __init__(self, O, leaf: int, rotation: bool, tree: int = 0):
        self.O = O
        self.leaf = leaf
        self.rotation = rotation
        self.tree = tree
        f1, f2 = O.fanouts(leaf, tree)
        self.lower1 = f1 * leaf
        self.lower2 = f2 * f1 * leaf
        self.salts = {}

    def salt(self, level):
        if level not in self.salts:
            self.salts[level] = self.O.salt(level)
        return self.salts[level]

    def h(self, lo, level, s, m):
        return self.O.mix64((int(lo) + self.salt(level) + s) & M64) % m

    def level(self, m, depth):
        if m <= self.leaf:
            return 0
        if m <= self.lower1:
            return 1
        if m <= self.lower2:
            return 2
        return 3 + depth

    def split_ok(self, lo, m, depth, s, parts):
        lev = self.level(m, depth)
        counts = [0] * len(parts)
        for x in lo:
            p = self.h(x, lev, s, m)
            counts[self.child(m, parts, p)] += 1
        return counts == parts

    def child(self, m, parts, pos):
        if m > self.lower2:
            return 0 if pos < parts[0] else 1
        unit = self.leaf if m <= self.lower1 else self.lower1
        return pos // unit

    def leaf_ok(self, lo, hi, m, x):
        if not self.rotation:
            return sorted(self.h(v, 0, x, m) for v in lo) == list(range(m))
        r = x % m
        seed = x - r
        pos = []
        for v, w in zip(lo, hi):
            p = self.h(v, 0, seed, m)
            pos.append((p + r) % m if int(w) & 1 else p)
        return sorted(pos) == list(range(m))

    def check_bucket(self, lo, hi, values, max_brute=20000):
        """values: this bucket's stored values in preorder.  Returns nodes checked."""
        it = iter(values)
        n = self._node(list(lo), list(hi), len(lo), 0, it, max_brute)
        rest = list(it)
        assert not rest, f"{len(rest)} values left over"
        return n

    def _node(self, lo, hi, m, depth, it, max_brute):
        if m <= 1:
            return 0
        x = int(next(it))
        if m <= self.leaf:
            assert self.leaf_ok(lo, hi, m, x), "stored leaf value is not a bijection"
            if x <= max_brute:
                for y in range(x):
                    assert not self.leaf_ok(lo, hi, m, y), f"smaller leaf value {y} < {x} works"
            return 1
        parts = self.O.parts(self.leaf, m, self.tree)
        assert self.split_ok(lo, m, depth, x, parts), "stored split does not split"
        if x <= max_brute:
            for y in range(x):
                assert not self.split_ok(lo, m, depth, y, parts), f"smaller split {y} < {x} works"
        lev = self.level(m, depth)
        groups = [[] for _ in parts]
        for v, w in zip(lo, hi):
            groups[self.child(m, parts, self.h(v, lev, x, m))].append((v, w))
        n = 1
        for g, p in zip(groups, parts):
            assert len(g) == p
            n += self._node([a for a, _ in g], [b for _, b in g], p, depth + 1, it, max_brute)
        return n


def group_by_bucket(O, keys: np.ndarray, nb: int):
    """(hi, lo) of every key grouped by bucket, via the oracle's fingerprint."""
    hi, lo = O.fingerprint(keys)
    b = np.array([O.bucket_of(int(h), nb) for h in hi], dtype=np.int64)
    groups = {}
    for i in range(len(keys)):
        groups.setdefault(int(b[i]), []).append(i)
    return hi, lo, groups


BLOB_MAGIC = int.from_bytes(b"RMPFPH01", "little")


def oracle_blob(o, leaf: int, bucket: int, key_bytes: int, bij: int, tree: int) -> bytes:
    """The serialised form (16 header words, Golomb-Rice words, Elias-Fano
    words, as include/mphf.h lays it out) of a function the oracle built.
    Elias-Fano word counts of a sequence of k values ending at U with L low
    bits: ceil(k L / 64) low words and ceil(((U >> L) + k) / 64) high words."""
    k = o.nb + 1

    def dims(last, L):
        return (k * L + 63) // 64, ((last >> L) + k + 63) // 64

    l0, h0 = dims(o.n, o.ef_L[0])
    l1, h1 = dims(o.gr_bits, o.ef_L[1])
    assert l0 + h0 + l1 + h1 == len(o.ef)
    head = np.array([BLOB_MAGIC, o.n, o.nb, leaf | (tree << 16), bucket, key_bytes, bij, o.gr_bits,
                     len(o.gr), len(o.ef), o.ef_L[0], o.ef_L[1], l0, h0, l1, h1], np.uint64)
    return head.tobytes() + o.gr.astype(np.uint64).tobytes() + o.ef.astype(np.uint64).tobytes()


def read_serialised_fixture(name: str = "serialised_l8_rotation.txt"):
    """(params, blob bytes, keys, values) of a serialised-function fixture."""
    params, words, pairs = {}, [], []
    section = None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line.startswith("# params"):
                params = {k: int(v) for k, v in (t.split("=") for t in line.split()[2:])}
                continue
            if not line or line.startswith("#"):
                continue
            if line.startswith(("words", "keys")):
                section = line.split()[0]
                continue
            if section == "words":
                words.append(int(line, 16))
            else:
                k, v = line.split()
                pairs.append((int(k, 16), int(v)))
    blob = np.array(words, np.uint64).tobytes()
    keys = np.array([k for k, _ in pairs], np.uint64)
    values = np.array([v for _, v in pairs], np.uint64)
    return params, blob, keys, values
