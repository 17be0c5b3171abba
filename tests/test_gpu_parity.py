"""GPU parity: the CUDA build against the CPU oracle, bit for bit.

Stored values (split seeds, leaf seeds, k*m + r of rotation leaves), bucket
offsets, Golomb-Rice words, Elias-Fano words and the trial statistics must be
identical; queries must agree and form a bijection onto [0, n).  Small cases
span several buckets and ragged tails; the large workloads are compared on a
seeded sample of buckets, in the launch shape the benchmark uses, and checked
for bijectivity over every key on the device.
"""
import os

import numpy as np
import pytest

from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W
from test_oracle_search import _keys_with_fingerprints

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_09562_b300 import build
    build.build()
    M.lib()
    return t


def to_dev(torch, keys: np.ndarray):
    if keys.ndim == 1:
        return torch.from_numpy(keys.view(np.int64)).cuda()
    return torch.from_numpy(np.ascontiguousarray(keys)).cuda()


def assert_same_function(o, g, keys_np, dkeys, full=True):
    a = g.host_arrays()
    assert g.info.n == o.n and g.info.nb == o.nb and g.info.n_nodes == o.n_nodes
    assert np.array_equal(a["cum_keys"], o.cum_keys)
    assert np.array_equal(a["node_off"], o.node_off)
    assert np.array_equal(a["values"], o.values)
    assert np.array_equal(a["bit_pos"], o.bit_pos)
    assert g.info.gr_bits == o.gr_bits
    assert np.array_equal(a["gr"], o.gr)
    assert np.array_equal(a["ef"], o.ef)
    st = g.stats()
    for k in ("leaf", "lower1", "lower2", "upper"):
        assert st[k] == o.stats[k], k
    if full and len(keys_np):
        q = g.query(dkeys).cpu().numpy().view(np.uint64)
        assert np.array_equal(q, o.query(keys_np))
    assert g.verify(dkeys) == 0


SMALL = [(8, 100, False, 8, n) for n in (1, 2, 7, 8, 9, 100, 307, 5000)] + [
    (8, 100, True, 16, 3000), (12, 1000, True, 8, 4321), (12, 57, True, 16, 3000),
    (16, 2000, True, 8, 2500), (16, 300, True, 8, 3001), (5, 7, True, 8, 3000),
    (2, 5, True, 8, 500), (3, 40, False, 8, 800), (10, 250, True, 16, 2600),
    (20, 3, True, 8, 700), (7, 3000, True, 8, 6100), (16, 17, False, 8, 400),
    # more than 8192 buckets: the global-atomic bucket sort instead of the two-level one
    (8, 10, True, 8, 100_000), (5, 5, False, 16, 60_000),
]


@pytest.mark.parametrize("leaf,bucket,rotation,kb,n", SMALL)
def test_small_builds_match_the_oracle(torch, orc, leaf, bucket, rotation, kb, n):
    keys = W.random_keys(n, kb, 1000 + 7 * n + leaf)
    o = orc.build_mphf(keys, leaf, bucket, rotation, threads=THREADS)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, leaf, bucket, rotation)
    assert_same_function(o, g, keys, dkeys)


def test_empty_build(torch, orc):
    keys = np.zeros(0, np.uint64)
    o = orc.build_mphf(keys, 8, 100, True)
    g = M.MPHF.build(to_dev(torch, keys), 8, 100, True)
    assert g.info.n == 0 and g.info.nb == 0 and g.info.n_nodes == 0
    assert np.array_equal(g.host_arrays()["ef"], o.ef)


@pytest.mark.parametrize("threads,blocks", [(64, 1), (128, 2), (512, 1), (256, 0)])
def test_launch_shape_does_not_change_the_result(torch, orc, threads, blocks):
    keys = W.distinct_u64(20000, 77)
    o = orc.build_mphf(keys, 12, 500, True, threads=THREADS)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, 12, 500, True, threads_per_block=threads, blocks_per_sm=blocks)
    assert_same_function(o, g, keys, dkeys)


def test_host_build_equals_device_build(torch, orc):
    keys = W.distinct_bytes16(40000, 78)
    dkeys = to_dev(torch, keys)
    g1 = M.MPHF.build(dkeys, 8, 100, True)
    g2 = M.MPHF.build_host(keys, 8, 100, True)
    a1, a2 = g1.host_arrays(), g2.host_arrays()
    for k in a1:
        assert np.array_equal(a1[k], a2[k]), k
    s = g2.serialize()
    words = np.frombuffer(s[128:], np.uint64)
    assert np.array_equal(words[: g2.info.gr_words], a2["gr"])
    assert np.array_equal(words[g2.info.gr_words:], a2["ef"])


def test_duplicates_are_refused(torch, orc):
    keys = W.distinct_u64(3000, 79)
    keys[10] = keys[2000]
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build(to_dev(torch, keys), 8, 100, True)
    assert e.value.code == M.EDUPLICATE
    with pytest.raises(orc.OracleError) as e2:
        orc.build_mphf(keys, 8, 100, True)
    assert e2.value.code == orc.EDUPLICATE


def test_equal_lo_words_are_refused(torch, orc):
    rng = np.random.default_rng(80)
    his = [int(x) for x in rng.integers(0, 2**62, 300, dtype=np.int64)]
    los = [int(x) for x in rng.integers(0, 2**62, 300, dtype=np.int64)]
    los[3] = los[250]
    his[250] = his[3] ^ 1  # same bucket, different rotation bit
    keys = _keys_with_fingerprints(orc, his, los)
    for rotation in (False, True):
        with pytest.raises(M.MPHFError) as e:
            M.MPHF.build(to_dev(torch, keys), 8, 100, rotation)
        assert e.value.code == M.EDUPLICATE


def test_oversized_bucket_is_refused(torch, orc):
    rng = np.random.default_rng(81)
    n = 4097
    his = [int(x) for x in rng.integers(0, 2**63 - 1, n, dtype=np.int64)]
    los = [int(x) for x in rng.integers(0, 2**63 - 1, n, dtype=np.int64)]
    keys = _keys_with_fingerprints(orc, his, los)
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build(to_dev(torch, keys), 8, 3000, True)
    assert e.value.code == M.EBUCKET


@pytest.mark.parametrize("rotation", [False, True])
def test_search_cap_and_precedence(torch, orc, rotation):
    keys = W.distinct_u64(2000, 82)
    for maxv in (3, 40):
        with pytest.raises(M.MPHFError) as e:
            M.MPHF.build(to_dev(torch, keys), 8, 100, rotation, max_value=maxv)
        assert e.value.code == M.ESEARCH_LIMIT
        with pytest.raises(orc.OracleError) as e2:
            orc.build_mphf(keys, 8, 100, rotation, max_value=maxv)
        assert e2.value.code == orc.ESEARCH_LIMIT
    keys[5] = keys[6]
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build(to_dev(torch, keys), 8, 100, rotation, max_value=3)
    assert e.value.code == M.EDUPLICATE


def test_large_cap_is_not_hit(torch, orc):
    """A cap just above every stored value still succeeds with the same values."""
    keys = W.distinct_u64(5000, 83)
    o = orc.build_mphf(keys, 8, 100, True)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, 8, 100, True, max_value=int(o.values.max()))
    assert_same_function(o, g, keys, dkeys)


def test_plain_l8_workload_full(torch, orc):
    w = W.WORKLOADS["plain_l8"]
    keys = W.keys_for(w)
    o = orc.build_mphf(keys, w.leaf, w.bucket, w.rotation, threads=THREADS)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, w.leaf, w.bucket, w.rotation)
    assert_same_function(o, g, keys, dkeys)


def _sampled_parity(torch, orc, name, count):
    w = W.WORKLOADS[name]
    keys = W.keys_for(w)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, w.leaf, w.bucket, w.rotation)
    a = g.host_arrays()
    nb = g.info.nb
    sample = W.sample_buckets(nb, count, w.seed)
    vals, counts, _ = orc.build_sample(keys, w.leaf, w.bucket, w.rotation, sample, threads=THREADS)
    off = 0
    for b, c in zip(sample, counts):
        b = int(b)
        want = vals[off:off + int(c)]
        got = a["values"][int(a["node_off"][b]):int(a["node_off"][b + 1])]
        assert np.array_equal(got, want), f"bucket {b}"
        off += int(c)
    # bucket sizes equal the oracle's recount; the whole function is a bijection
    hi, _ = orc.fingerprint(keys)
    h, l = hi >> np.uint64(32), hi & np.uint64(0xFFFFFFFF)
    bidx = ((h * np.uint64(nb) + ((l * np.uint64(nb)) >> np.uint64(32))) >> np.uint64(32)).astype(np.int64)
    counts_all = np.bincount(bidx, minlength=nb)
    assert np.array_equal(np.diff(a["cum_keys"]).astype(np.int64), counts_all)
    assert g.verify(dkeys) == 0
    return g


def test_rot_l12_workload_full(torch, orc):
    """The whole 10^6-key, 16-byte-key workload with l = 12, b = 1000 and
    rotation fitting, in the benchmark's launch shape: every node value, the
    offsets, the Golomb-Rice and Elias-Fano words and the statistics equal the
    oracle's full build, and every key queries to the oracle's value."""
    w = W.WORKLOADS["rot_l12"]
    keys = W.keys_for(w)
    o = orc.build_mphf(keys, w.leaf, w.bucket, w.rotation, threads=THREADS)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, w.leaf, w.bucket, w.rotation)
    assert_same_function(o, g, keys, dkeys)


def test_rot_l16_workload_sampled(torch, orc):
    """The 10^7-key l = 16, b = 2000 workload: a seeded sample of 50 buckets
    (1 % of them) node by node against the oracle, bucket sizes recounted,
    bijectivity over all keys."""
    _sampled_parity(torch, orc, "rot_l16", 50)


OUTSIDE = [  # (leaf, bucket, leaf method, tree, key bytes, n)
    (8, 100, M.PLAIN, M.TREE_RECSPLIT, 8, 5000),
    (12, 1000, M.ROTATION, M.TREE_RECSPLIT, 16, 20000),
    (16, 300, M.ROTATION, M.TREE_RECSPLIT, 8, 3000),
    (24, 2000, M.SHOCKHASH, M.TREE_FANOUT2, 8, 20000),
    (12, 300, M.SHOCKHASH, M.TREE_RECSPLIT, 8, 9000),
    (10, 500, M.PLAIN, M.TREE_FANOUT2, 16, 8000),
    (5, 1, M.ROTATION, M.TREE_RECSPLIT, 8, 50),  # about a third of the buckets empty
]


@pytest.mark.parametrize("leaf,bucket,bij,tree,kb,n", OUTSIDE)
def test_keys_outside_the_set_walk_like_the_oracle(torch, orc, leaf, bucket, bij, tree, kb, n):
    """Section 2.2, "Query": outside S the value is arbitrary, but the walk
    is the same definition on both sides (bucket, Elias-Fano lookups, one
    decoded value and child per level, the leaf's position; empty and
    one-key buckets return their key offset), so every value must agree."""
    keys = W.random_keys(n, kb, 31 * n + leaf)
    o = orc.build_mphf(keys, leaf, bucket, bij, threads=THREADS, tree=tree)
    g = M.MPHF.build(to_dev(torch, keys), leaf, bucket, bij, tree=tree)
    other = W.random_keys(100_000, kb, 977 + leaf + kb)
    got = g.query(to_dev(torch, other)).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, o.query(other))


@pytest.mark.parametrize("leaf,rotation", [(8, True), (12, False), (16, True)])
def test_largest_bucket_matches_the_oracle(torch, orc, leaf, rotation):
    """A bucket of exactly MAX_BUCKET (4096) keys, the largest a build accepts
    (reading R12): all keys' hi words below 2^63, so with n = 4096 and b = 3000
    (two buckets) every key lands in bucket 0.  Its whole tree, including the
    fanout-2 levels above the lower aggregation levels, equals the oracle's."""
    rng = np.random.default_rng(90 + leaf)
    n = M.MAX_BUCKET
    his = [int(x) for x in rng.integers(0, 2**63 - 1, n, dtype=np.int64)]
    los = [int(x) for x in rng.integers(0, 2**63 - 1, n, dtype=np.int64)]
    keys = _keys_with_fingerprints(orc, his, los)
    o = orc.build_mphf(keys, leaf, 3000, rotation, threads=THREADS)
    assert int(o.cum_keys[1]) == n  # one full bucket, one empty
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, leaf, 3000, rotation)
    assert g.info.max_bucket == n
    assert_same_function(o, g, keys, dkeys)
