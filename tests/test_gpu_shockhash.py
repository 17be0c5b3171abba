"""GPU parity of ShockHash leaves (Appendix C) against the CPU oracle.

Stored words (split seeds; leaf seed with its retrieval vector in the bits
from 40 up), Golomb-Rice and Elias-Fano words and the trial statistics must
be identical; queries must agree and form a bijection.  Small cases span
several buckets, leaves of every size up to l and ragged tails; the large
workload is compared on a seeded sample of buckets in the benchmark's launch
shape, with the whole function checked for bijectivity on the device.
"""
import ctypes
import os

import numpy as np
import pytest

from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W
from test_gpu_parity import assert_same_function, to_dev

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


SMALL = [(8, 100, 8, n) for n in (1, 2, 3, 8, 9, 100, 5000)] + [
    (2, 5, 8, 500), (3, 40, 16, 800), (4, 30, 8, 3000), (5, 7, 8, 3000), (7, 3000, 8, 6100),
    (10, 250, 16, 2600), (12, 1000, 8, 4321), (12, 57, 16, 3000), (16, 2000, 8, 2500),
    (16, 300, 8, 3001), (16, 17, 16, 400), (20, 3, 8, 700), (24, 2, 8, 300), (24, 30, 16, 500),
    # more than 8192 buckets: the global-atomic bucket sort
    (8, 10, 8, 100_000),
]


@pytest.mark.parametrize("leaf,bucket,kb,n", SMALL)
def test_small_shockhash_builds_match_the_oracle(torch, orc, leaf, bucket, kb, n):
    keys = W.random_keys(n, kb, 3000 + 7 * n + leaf)
    o = orc.build_mphf(keys, leaf, bucket, orc.SHOCKHASH, threads=THREADS)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, leaf, bucket, M.SHOCKHASH)
    assert g.info.leaf_bijection == M.SHOCKHASH
    assert_same_function(o, g, keys, dkeys)


@pytest.mark.parametrize("threads,blocks", [(64, 1), (256, 2), (512, 0)])
def test_launch_shape_does_not_change_the_shockhash_result(torch, orc, threads, blocks):
    keys = W.distinct_u64(20000, 3077)
    o = orc.build_mphf(keys, 12, 500, orc.SHOCKHASH, threads=THREADS)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, 12, 500, M.SHOCKHASH, threads_per_block=threads, blocks_per_sm=blocks)
    assert_same_function(o, g, keys, dkeys)


def test_shockhash_search_cap_and_duplicates(torch, orc):
    keys = W.distinct_u64(2000, 3082)
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build(to_dev(torch, keys), 8, 100, M.SHOCKHASH, max_value=2)
    assert e.value.code == M.ESEARCH_LIMIT
    with pytest.raises(orc.OracleError) as e2:
        orc.build_mphf(keys, 8, 100, orc.SHOCKHASH, max_value=2)
    assert e2.value.code == orc.ESEARCH_LIMIT
    keys[5] = keys[6]
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build(to_dev(torch, keys), 8, 100, M.SHOCKHASH, max_value=2)
    assert e.value.code == M.EDUPLICATE


def test_host_build_and_serialised_words(torch, orc):
    keys = W.distinct_bytes16(30000, 3083)
    g1 = M.MPHF.build(to_dev(torch, keys), 12, 1000, M.SHOCKHASH)
    g2 = M.MPHF.build_host(keys, 12, 1000, M.SHOCKHASH)
    a1, a2 = g1.host_arrays(), g2.host_arrays()
    for k in a1:
        assert np.array_equal(a1[k], a2[k]), k
    o = orc.build_mphf(keys, 12, 1000, orc.SHOCKHASH, threads=THREADS)
    words = np.frombuffer(g2.serialize()[128:], np.uint64)
    assert np.array_equal(words[: g2.info.gr_words], o.gr)
    assert np.array_equal(words[g2.info.gr_words:], o.ef)


def test_batch_mixes_leaf_methods(torch, orc):
    """One persistent search over builds with plain, rotation and ShockHash
    leaves: each equals its own build and the oracle."""
    specs = [(5000, 8, M.PLAIN), (7000, 12, M.ROTATION), (6000, 16, M.SHOCKHASH),
             (3000, 8, M.SHOCKHASH), (0, 8, M.SHOCKHASH), (1, 12, M.SHOCKHASH)]
    keys = [W.distinct_u64(n, 3090 + i) for i, (n, _, _) in enumerate(specs)]
    dkeys = [to_dev(torch, k) for k in keys]
    descs = (M.BuildDesc * len(specs))()
    for i, ((n, leaf, bij), dk) in enumerate(zip(specs, dkeys)):
        descs[i] = M.BuildDesc(dk.data_ptr() if n else None, n, leaf, 500, 8, bij, 0, 0, 0)
    outs = (ctypes.c_void_p * len(specs))()
    sts = (ctypes.c_int * len(specs))()
    stream = torch.cuda.current_stream().cuda_stream
    assert M.lib().mphf_build_batch(descs, len(specs), stream, outs, sts) == M.OK
    for i, ((n, leaf, bij), k, dk) in enumerate(zip(specs, keys, dkeys)):
        built = M.MPHF(outs[i])
        alone = M.MPHF.build(dk, leaf, 500, bij)
        a, b = built.host_arrays(), alone.host_arrays()
        for name in a:
            assert np.array_equal(a[name], b[name]), (i, name)
        if n:
            o = orc.build_mphf(k, leaf, 500, bij, threads=THREADS)
            assert np.array_equal(a["values"], o.values)
            assert np.array_equal(a["gr"], o.gr)
            assert built.verify(dk) == 0


def test_shock_l16_workload_sampled(torch, orc):
    w = W.WORKLOADS["shock_l16"]
    keys = W.keys_for(w)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, w.leaf, w.bucket, w.rotation)
    a = g.host_arrays()
    sample = W.sample_buckets(g.info.nb, max(4, min(16, THREADS)), w.seed)
    vals, counts, _ = orc.build_sample(keys, w.leaf, w.bucket, w.rotation, sample, threads=THREADS)
    off = 0
    for b, c in zip(sample, counts):
        b = int(b)
        got = a["values"][int(a["node_off"][b]):int(a["node_off"][b + 1])]
        assert np.array_equal(got, vals[off:off + int(c)]), f"bucket {b}"
        off += int(c)
    assert g.verify(dkeys) == 0
