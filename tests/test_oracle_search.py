"""Oracle pins: the brute-force searches.

* Brute force on tiny inputs: every stored value works and no smaller value
  does, for splits, plain leaves and rotation leaves (Section 2.2,
  "Bijections"; Section 4; Section 5.1 on keeping the smallest stored number).
* Statistics: mean trial counts match the closed forms (brute-force leaf
  l^l/l!, multinomial splits, rotation fitting by exact enumeration) and the
  hash-evaluation ratio of the Appendix C figure on hash function evaluations.
* Error paths: duplicates, the search cap, bad parameters, oversized buckets.
"""
import math

import numpy as np
import pytest

from helpers import M64, NaiveChecker, golden_pairs, group_by_bucket
from paper_2212_09562_b300 import workloads as W
from test_oracle_probability import exact_rotation_success


@pytest.mark.parametrize("leaf,bucket,rotation,kb,n", [
    (4, 30, False, 8, 200), (4, 30, True, 8, 200), (5, 60, True, 16, 300),
    (6, 100, False, 8, 260), (6, 100, True, 16, 260), (3, 50, True, 8, 150),
    (2, 20, True, 8, 80), (2, 20, False, 8, 80),
])
def test_every_node_is_minimal_by_brute_force(orc, leaf, bucket, rotation, kb, n):
    keys = W.random_keys(n, kb, 100 + leaf)
    h = orc.build_mphf(keys, leaf, bucket, rotation)
    hi, lo, groups = group_by_bucket(orc, keys, h.nb)
    chk = NaiveChecker(orc, leaf, rotation)
    checked = 0
    for b in range(h.nb):
        idx = groups.get(b, [])
        vals = h.values[int(h.node_off[b]):int(h.node_off[b + 1])]
        checked += chk.check_bucket(lo[idx], hi[idx], vals)
    assert checked == h.n_nodes and checked > 10


def test_rotation_value_is_smallest_over_seed_and_rotation(orc):
    """A leaf where a larger rotation of an earlier seed must beat a later seed:
    the naive checker walks every k*m + r below the stored value."""
    rng = np.random.default_rng(8)
    chk = NaiveChecker(orc, 7, True)
    for _ in range(60):
        lo = rng.integers(0, 2**63, 7, dtype=np.int64).astype(np.uint64)
        hi = rng.integers(0, 2, 7).astype(np.uint64)
        rc, x, trials, evals = orc.node_search(7, True, lo, hi)
        assert rc == 0
        assert chk.leaf_ok(list(lo), list(hi), 7, x)
        assert all(not chk.leaf_ok(list(lo), list(hi), 7, y) for y in range(x))
        assert trials == x // 7 + 1 and evals == 7 * trials


def _mean_trials(orc, leaf, rotation, m, count, seed, depth=0):
    rng = np.random.default_rng(seed)
    t = []
    for _ in range(count):
        lo = rng.integers(0, 2**63, m, dtype=np.int64).astype(np.uint64) * np.uint64(2) + \
            rng.integers(0, 2, m).astype(np.uint64)
        hi = rng.integers(0, 2, m).astype(np.uint64)
        rc, x, trials, evals = orc.node_search(leaf, rotation, lo, hi, depth)
        assert rc == 0 and evals == trials * m
        t.append(trials)
    t = np.asarray(t, float)
    return t.mean(), t.std(ddof=1) / math.sqrt(len(t))


def test_plain_leaf_trials_match_l_to_the_l_over_l_factorial(orc):
    mean, se = _mean_trials(orc, 8, False, 8, 4000, 21)
    expected = 8**8 / math.factorial(8)
    assert abs(mean - expected) < 4.5 * se, (mean, expected, se)


@pytest.mark.parametrize("leaf,count", [(8, 6000), (12, 1500), (16, 800)])
def test_rotation_leaf_trials_match_exact_enumeration(orc, leaf, count):
    m = leaf
    expected = sum(math.comb(m, a) * 2.0**-m / exact_rotation_success(m, a) for a in range(m + 1))
    mean, se = _mean_trials(orc, leaf, True, m, count, 22 + leaf)
    assert abs(mean - expected) < 4.5 * se, (mean, expected, se)
    if leaf == 8:
        assert expected == pytest.approx(56.481, rel=1e-4)
    if leaf == 12:
        assert expected == pytest.approx(1575.40, rel=1e-4)
    if leaf == 16:  # the benchmark's leaf size
        assert expected == pytest.approx(55239.48, rel=1e-5)


@pytest.mark.parametrize("leaf,m,depth,count", [(8, 32, 0, 3000), (8, 96, 0, 1500), (8, 20, 0, 3000),
                                                (8, 200, 0, 2500), (8, 200, 2, 2500)])
def test_split_trials_match_the_multinomial(orc, leaf, m, depth, count):
    expected = 1 / orc.split_success(leaf, m)
    mean, se = _mean_trials(orc, leaf, False, m, count, 30 + m + depth, depth)
    assert abs(mean - expected) < 4.5 * se, (mean, expected, se)


def test_hash_evaluation_ratio_matches_the_appendix_figure(orc):
    """Rotation fitting hashes all m keys per k; brute force stops a trial at
    the first collision.  The ratio of mean evaluations reproduces the
    paper's measured curve at l = 8 (0.2554) within sampling error."""
    paper = dict(golden_pairs("fig_hash_evals_rotation.txt"))
    m = 8
    rng = np.random.default_rng(40)
    rot, brute = [], []
    for _ in range(5000):
        lo = rng.integers(0, 2**63, m, dtype=np.int64).astype(np.uint64)
        hi = rng.integers(0, 2, m).astype(np.uint64)
        rc, x, trials, evals = orc.node_search(m, True, lo, hi)
        rot.append(evals)
        brute.append(orc.leaf_plain_early_exit(lo)[1])
    ratio = np.mean(rot) / np.mean(brute)
    # expected evaluations of one brute-force trial that stops at a collision
    e_trial = sum(math.prod(1 - i / m for i in range(j)) for j in range(m))
    e_rot = sum(math.comb(m, a) * 2.0**-m / exact_rotation_success(m, a) for a in range(m + 1))
    model = (m * e_rot) / (m**m / math.factorial(m) * e_trial)
    assert model == pytest.approx(paper[8], rel=0.01)
    assert ratio == pytest.approx(paper[8], rel=0.08), ratio


def test_duplicate_keys_are_refused(orc):
    keys = W.distinct_u64(500, 50)
    keys[17] = keys[300]
    with pytest.raises(orc.OracleError) as e:
        orc.build_mphf(keys, 8, 100, True)
    assert e.value.code == orc.EDUPLICATE


def _keys_with_fingerprints(orc, his, los):
    """16-byte keys whose fingerprints are the given (hi, lo): invert the Feistel rounds."""
    G = 0x9E3779B97F4A7C15
    out = np.zeros((len(his), 16), np.uint8)
    for i, (h, l) in enumerate(zip(his, los)):
        t1 = l ^ orc.mix64((h + 3 * G) & M64)
        w0 = h ^ orc.mix64((t1 + 2 * G) & M64)
        w1 = t1 ^ orc.mix64((w0 + G) & M64)
        out[i, :8] = np.frombuffer(int(w0).to_bytes(8, "little"), np.uint8)
        out[i, 8:] = np.frombuffer(int(w1).to_bytes(8, "little"), np.uint8)
    return out


def test_equal_lo_words_in_one_bucket_are_refused(orc):
    """Different keys whose fingerprints share the lo word can never be
    separated by any seed: the build refuses them as duplicates."""
    rng = np.random.default_rng(51)
    his = [int(x) for x in rng.integers(0, 2**62, 40, dtype=np.int64)]
    los = [int(x) for x in rng.integers(0, 2**62, 40, dtype=np.int64)]
    los[5] = los[9]
    keys = _keys_with_fingerprints(orc, his, los)
    hi, lo = orc.fingerprint(keys)
    assert [int(v) for v in lo] == los and [int(v) for v in hi] == his
    with pytest.raises(orc.OracleError) as e:
        orc.build_mphf(keys, 8, 100, True)
    assert e.value.code == orc.EDUPLICATE


def test_oversized_bucket_is_refused(orc):
    rng = np.random.default_rng(52)
    n = 4097
    his = [int(x) for x in rng.integers(0, 2**63 - 1, n, dtype=np.int64)]  # all in bucket 0 of 2
    los = [int(x) for x in rng.integers(0, 2**63 - 1, n, dtype=np.int64)]
    keys = _keys_with_fingerprints(orc, his, los)
    with pytest.raises(orc.OracleError) as e:
        orc.build_mphf(keys, 8, 3000, True)
    assert e.value.code == orc.EBUCKET


def test_search_cap(orc):
    keys = W.distinct_u64(2000, 53)
    with pytest.raises(orc.OracleError) as e:
        orc.build_mphf(keys, 8, 100, True, max_value=3)
    assert e.value.code == orc.ESEARCH_LIMIT
    # duplicates take precedence over the search cap
    keys[5] = keys[6]
    with pytest.raises(orc.OracleError) as e:
        orc.build_mphf(keys, 8, 100, True, max_value=3)
    assert e.value.code == orc.EDUPLICATE


def test_bad_parameters(orc):
    keys = W.distinct_u64(100, 54)
    for leaf, bucket in [(1, 100), (25, 100), (8, 0), (8, 3001)]:
        with pytest.raises(orc.OracleError) as e:
            orc.build_mphf(keys, leaf, bucket, True)
        assert e.value.code == orc.EINVAL


def test_threads_do_not_change_results(orc):
    keys = W.distinct_u64(20000, 55)
    a = orc.build_mphf(keys, 8, 100, True, threads=1)
    b = orc.build_mphf(keys, 8, 100, True, threads=5)
    assert np.array_equal(a.values, b.values) and np.array_equal(a.gr, b.gr)
    assert np.array_equal(a.ef, b.ef) and a.stats == b.stats


def test_sampled_buckets_match_the_full_build(orc):
    keys = W.distinct_u64(30000, 56)
    full = orc.build_mphf(keys, 8, 500, True)
    sample = np.array([3, 17, 59, 0], np.uint64)
    vals, counts, _ = orc.build_sample(keys, 8, 500, True, sample, threads=2)
    off = 0
    for b, c in zip(sample, counts):
        b = int(b)
        want = full.values[int(full.node_off[b]):int(full.node_off[b + 1])]
        assert np.array_equal(vals[off:off + int(c)], want)
        off += int(c)
