"""Oracle pins: hash function, fingerprint, bucket assignment.

The paper asks only for a high-quality initial hash (Section 2.2, "Splitting
Trees"; Section 6 uses random 128-bit master hash codes).  The hash chosen is
the SplitMix64 output function, pinned against the generator's published
outputs; the fingerprint is a Feistel network over it, pinned by inverting it.
"""
import numpy as np

from helpers import M64, golden_hex
from paper_2212_09562_b300 import workloads as W

G = 0x9E3779B97F4A7C15


def test_mix64_matches_splitmix64_reference_outputs(orc):
    expected = golden_hex("splitmix64_seed0.txt")
    got = [orc.mix64(((i + 1) * G) & M64) for i in range(len(expected))]
    assert got == expected


def test_mix64_is_a_bijection_on_a_sample(orc):
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 2**63, 20000, dtype=np.int64).astype(np.uint64)
    ys = {orc.mix64(int(x)) for x in xs}
    assert len(ys) == len(set(int(x) for x in xs))


def _inverse_feistel(orc, hi, lo):
    t1 = lo ^ orc.mix64((hi + 3 * G) & M64)
    w0 = hi ^ orc.mix64((t1 + 2 * G) & M64)
    w1 = t1 ^ orc.mix64((w0 + G) & M64)
    return w0, w1


def test_fingerprint_inverts_for_8_byte_keys(orc):
    keys = W.distinct_u64(2000, 11)
    hi, lo = orc.fingerprint(keys)
    for k, h, l in zip(keys, hi, lo):
        w0, w1 = _inverse_feistel(orc, int(h), int(l))
        assert (w0, w1) == (int(k), 0)


def test_fingerprint_inverts_for_16_byte_keys(orc):
    keys = W.distinct_bytes16(2000, 12)
    hi, lo = orc.fingerprint(keys)
    words = keys.view("<u8").reshape(-1, 2)
    for (a, b), h, l in zip(words, hi, lo):
        assert _inverse_feistel(orc, int(h), int(l)) == (int(a), int(b))


def test_8_byte_key_equals_16_byte_key_with_zero_high_word(orc):
    keys = W.distinct_u64(500, 13)
    wide = np.zeros((500, 16), np.uint8)
    wide[:, :8] = keys.view(np.uint8).reshape(-1, 8)
    a = orc.fingerprint(keys)
    b = orc.fingerprint(wide)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_fingerprints_distinct_on_a_million_keys(orc):
    keys = W.distinct_u64(1_000_000, 14)
    hi, lo = orc.fingerprint(keys)
    fp = np.stack([hi, lo], axis=1).view(np.dtype((np.void, 16))).reshape(-1)
    assert len(np.unique(fp)) == len(keys)


def test_bucket_is_monotone_and_in_range(orc):
    nb = 5000
    his = sorted(int(x) for x in np.random.default_rng(5).integers(0, 2**63, 3000, dtype=np.int64))
    his = [0, 1] + [2 * h for h in his] + [M64]
    bs = [orc.bucket_of(h, nb) for h in his]
    assert bs == sorted(bs)
    assert bs[0] == 0 and bs[-1] == nb - 1
    assert all(0 <= b < nb for b in bs)
    # equal-width ranges of the 64-bit space map to consecutive buckets
    for b in (0, 1, 1234, nb - 1):
        lo_edge = -(-(b << 64) // nb)  # smallest hi of bucket b
        assert orc.bucket_of(lo_edge, nb) == b
        if lo_edge > 0:
            assert orc.bucket_of(lo_edge - 1, nb) == b - 1


def test_bucket_sizes_follow_the_mean(orc):
    keys = W.distinct_u64(200_000, 15)
    hi, _ = orc.fingerprint(keys)
    nb = 200
    counts = np.bincount([orc.bucket_of(int(h), nb) for h in hi], minlength=nb)
    assert counts.sum() == len(keys)
    # Poisson-like: mean 1000, standard deviation about 32
    assert abs(counts.mean() - 1000) < 1e-9
    assert counts.std() < 60 and counts.min() > 800 and counts.max() < 1200
