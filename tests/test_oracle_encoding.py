"""Oracle pins: Golomb-Rice and Elias-Fano encodings and the query.

* Golomb-Rice (Section 2.1; Section 2.2 "Representation"): a decoder written
  here reads each bucket's fixed parts (preorder) and unary parts back and
  recovers the stored values.
* Elias-Fano (Section 2.1): a decoder written here recovers the bucket prefix
  sums (checked against a recount of the bucket sizes) and the bucket bit
  positions; the size respects k(2 + log(U/k)) bits up to word rounding.
* Query (Section 2.2 "Query"): a bijection onto [0, n) for every build.
"""
import math

import numpy as np
import pytest

from paper_2212_09562_b300 import workloads as W


def bits_of(words, start, count):
    v = 0
    for i in range(count):
        p = start + i
        v |= ((int(words[p >> 6]) >> (p & 63)) & 1) << i
    return v


def ef_decode(words, k, last):
    L = int(math.floor(math.log2(last // k))) if last >= k else 0
    low_words = (k * L + 63) // 64
    high_words = ((last >> L) + k + 63) // 64
    low, high = words[:low_words], words[low_words:low_words + high_words]
    out = []
    i = 0
    for w in range(high_words):
        for b in range(64):
            if (int(high[w]) >> b) & 1:
                out.append(((w * 64 + b - i) << L) | bits_of(low, i * L, L))
                i += 1
    return out, low_words + high_words


def preorder_sizes(orc, leaf, m):
    if m <= 1:
        return []
    out = [m]
    if m > leaf:
        for p in orc.parts(leaf, m):
            out += preorder_sizes(orc, leaf, p)
    return out


@pytest.mark.parametrize("leaf,bucket,rotation,kb,n", [(8, 100, False, 8, 20000),
                                                       (8, 100, True, 16, 20000),
                                                       (12, 1000, True, 8, 6000),
                                                       (5, 7, True, 8, 3000)])
def test_golomb_rice_round_trip(orc, leaf, bucket, rotation, kb, n):
    keys = W.random_keys(n, kb, 60 + leaf)
    h = orc.build_mphf(keys, leaf, bucket, rotation)
    tau = orc.tau_table(leaf, rotation)
    for b in range(h.nb):
        m = int(h.cum_keys[b + 1] - h.cum_keys[b])
        sizes = preorder_sizes(orc, leaf, m)
        vals = h.values[int(h.node_off[b]):int(h.node_off[b + 1])]
        assert len(sizes) == len(vals)
        pos = int(h.bit_pos[b])
        fixed = []
        for s in sizes:
            fixed.append(bits_of(h.gr, pos, int(tau[s])))
            pos += int(tau[s])
        for s, f, v in zip(sizes, fixed, vals):
            zeros = 0
            while not (int(h.gr[pos >> 6]) >> (pos & 63)) & 1:
                zeros += 1
                pos += 1
            pos += 1
            assert (zeros << int(tau[s])) | f == int(v)
        assert pos == int(h.bit_pos[b + 1])
    assert int(h.bit_pos[-1]) == h.gr_bits
    assert len(h.gr) == (h.gr_bits + 63) // 64


@pytest.mark.parametrize("n,bucket", [(0, 100), (1, 100), (99, 100), (5000, 100), (20000, 7),
                                      (30000, 2000)])
def test_elias_fano_round_trip(orc, n, bucket):
    keys = W.distinct_u64(n, 70)
    h = orc.build_mphf(keys, 8, bucket, True)
    nb = (n + bucket - 1) // bucket
    assert h.nb == nb
    # bucket sizes recounted from the fingerprints
    hi, _ = orc.fingerprint(keys)
    counts = np.bincount([orc.bucket_of(int(x), nb) for x in hi], minlength=nb) if n else []
    cum = [0] + list(np.cumsum(counts)) if n else [0]
    assert [int(v) for v in h.cum_keys] == [int(c) for c in cum]
    k = nb + 1
    dec1, used1 = ef_decode(h.ef, k, int(h.cum_keys[-1]))
    assert dec1 == [int(v) for v in h.cum_keys]
    dec2, used2 = ef_decode(h.ef[used1:], k, int(h.bit_pos[-1]))
    assert dec2 == [int(v) for v in h.bit_pos]
    assert used1 + used2 == len(h.ef)
    for last in (int(h.cum_keys[-1]), int(h.bit_pos[-1])):
        bound = k * (2 + math.log2(max(last, 1) / k)) if last >= k else 2 * k + 1
        L = int(math.floor(math.log2(last // k))) if last >= k else 0
        assert k * L + (last >> L) + k <= bound + 1


@pytest.mark.parametrize("leaf,bucket,rotation,kb,n", [
    (8, 100, False, 8, 30000), (8, 100, True, 16, 30000), (12, 1000, True, 16, 20000),
    (16, 2000, True, 8, 2500), (2, 5, True, 8, 2000), (3, 10, False, 8, 2000),
    (8, 100, True, 8, 1), (8, 100, True, 8, 2), (8, 100, True, 8, 8), (8, 100, True, 8, 9),
    (24, 2, True, 8, 500), (20, 30, True, 16, 1000),
])
def test_query_is_a_bijection(orc, leaf, bucket, rotation, kb, n):
    keys = W.random_keys(n, kb, 80 + n % 97)
    h = orc.build_mphf(keys, leaf, bucket, rotation, threads=4)
    q = h.query(keys)
    assert np.array_equal(np.sort(q), np.arange(n, dtype=np.uint64))


def test_empty_build(orc):
    h = orc.build_mphf(np.zeros(0, np.uint64), 8, 100, True)
    assert h.n == 0 and h.nb == 0 and h.n_nodes == 0 and h.gr_bits == 0
    assert len(h.query(np.zeros(0, np.uint64))) == 0


def test_space_is_close_to_the_paper(orc):
    """Plausibility only (our parameter rule and directory are our own):
    l = 8, b = 100: 1.806 bits/key in the paper's query table;
    l = 16, b = 2000: 1.560 bits/key in its overall table."""
    keys = W.distinct_u64(50000, 90)
    h = orc.build_mphf(keys, 8, 100, False, threads=4)
    bits = (h.gr_bits + 64 * len(h.ef)) / h.n
    assert 1.70 < bits < 1.92, bits
    keys = W.distinct_u64(6000, 91)
    h = orc.build_mphf(keys, 16, 2000, True, threads=4)
    bits = (h.gr_bits + 64 * len(h.ef)) / h.n
    assert 1.50 < bits < 1.64, bits
