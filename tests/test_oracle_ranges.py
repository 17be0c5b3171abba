"""Oracle pin: building consecutive bucket ranges separately and joining
them gives the whole function (Section 5.2, "Multi-Threading": each thread
builds a consecutive range of buckets and produces local sequences that are
concatenated).  Node values, key / node / bit offsets and the Golomb-Rice
words of the joined ranges equal the single build's, for every way of
cutting nb buckets into ranges, including empty ranges; a key outside its
range is refused."""
import numpy as np
import pytest

from paper_2212_09562_b300 import workloads as W
from shard_ref import bucket_of_keys, concat_ranges, oracle_part

CASES = [  # (leaf, bucket, rotation, key bytes, n, cuts of [0, nb))
    (8, 100, True, 8, 5000, [0, 17, 18, 33, 50]),
    (8, 100, False, 16, 3000, [0, 0, 10, 30, 30]),
    (12, 300, True, 8, 9000, [0, 1, 29, 30]),
    (5, 7, 2, 8, 700, [0, 50, 100]),             # ShockHash leaves
    (16, 300, True, 8, 1500, [0, 1, 2, 3, 4, 5]),  # a range of one bucket each
]


@pytest.mark.parametrize("leaf,bucket,rotation,kb,n,cuts", CASES)
def test_ranges_join_to_the_whole_function(orc, leaf, bucket, rotation, kb, n, cuts):
    keys = W.random_keys(n, kb, 4400 + n + leaf)
    whole = orc.build_mphf(keys, leaf, bucket, rotation, threads=4)
    nb = whole.nb
    assert cuts[-1] == nb
    b = bucket_of_keys(orc, keys, nb)
    parts = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        sel = (b >= lo) & (b < hi)
        part = orc.build_range(keys[sel], n, leaf, bucket, rotation, lo, hi, threads=2)
        assert part.nb == hi - lo and part.n == int(sel.sum())
        parts.append(oracle_part(part))
    j = concat_ranges(parts)
    for name in ("cum_keys", "node_off", "bit_pos", "values", "gr"):
        assert np.array_equal(j[name], getattr(whole, name)), name
    assert j["gr_bits"] == whole.gr_bits


def test_key_outside_the_range_is_refused(orc):
    keys = W.distinct_u64(2000, 4500)
    nb = 20
    b = bucket_of_keys(orc, keys, nb)
    sel = b < 10
    sel[np.nonzero(~sel)[0][0]] = True  # one key of bucket >= 10
    with pytest.raises(orc.OracleError) as e:
        orc.build_range(keys[sel], 2000, 8, 100, True, 0, 10)
    assert e.value.code == orc.EINVAL
