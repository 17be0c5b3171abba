"""GPU parity of the fanout-2 splitting tree (Appendix C) against the oracle.

Every inner node splits in two, the left part a multiple of l; leaves may be
brute force, rotation fitting or ShockHash.  Small cases compare every word;
the large ShockHash workload (l = 24) is compared in full against the oracle,
which builds it in seconds, in the benchmark's launch shape.
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
F2 = M.TREE_FANOUT2


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_09562_b300 import build
    build.build()
    M.lib()
    return t


SMALL = [
    (8, 100, M.PLAIN, 8, 5000), (8, 2000, M.ROTATION, 16, 6000), (12, 1000, M.ROTATION, 8, 4321),
    (16, 2000, M.SHOCKHASH, 8, 9000), (24, 2000, M.SHOCKHASH, 16, 7000), (24, 3000, M.SHOCKHASH, 8, 6001),
    (20, 57, M.SHOCKHASH, 8, 3000), (2, 5, M.SHOCKHASH, 8, 500), (3, 40, M.ROTATION, 8, 800),
    (24, 7, M.SHOCKHASH, 8, 500), (8, 100, M.SHOCKHASH, 8, 1), (8, 100, M.SHOCKHASH, 8, 9),
    (24, 10, M.SHOCKHASH, 8, 100_000),  # more than 8192 buckets
]


@pytest.mark.parametrize("leaf,bucket,bij,kb,n", SMALL)
def test_small_fanout2_builds_match_the_oracle(torch, orc, leaf, bucket, bij, kb, n):
    keys = W.random_keys(n, kb, 4000 + 7 * n + leaf)
    o = orc.build_mphf(keys, leaf, bucket, bij, threads=THREADS, tree=orc.TREE_FANOUT2)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, leaf, bucket, bij, tree=F2)
    assert g.info.tree_shape == F2
    assert_same_function(o, g, keys, dkeys)


def test_batch_mixes_tree_shapes(torch, orc):
    specs = [(6000, 24, M.SHOCKHASH, F2), (5000, 16, M.SHOCKHASH, 0), (7000, 8, M.ROTATION, F2),
             (4000, 12, M.ROTATION, 0)]
    keys = [W.distinct_u64(n, 4100 + i) for i, (n, *_rest) in enumerate(specs)]
    dkeys = [to_dev(torch, k) for k in keys]
    descs = (M.BuildDesc * len(specs))()
    for i, ((n, leaf, bij, tree), dk) in enumerate(zip(specs, dkeys)):
        descs[i] = M.BuildDesc(dk.data_ptr(), n, leaf, 1000, 8, bij, 0, tree, 0)
    outs = (ctypes.c_void_p * len(specs))()
    sts = (ctypes.c_int * len(specs))()
    stream = torch.cuda.current_stream().cuda_stream
    assert M.lib().mphf_build_batch(descs, len(specs), stream, outs, sts) == M.OK
    for i, ((n, leaf, bij, tree), k, dk) in enumerate(zip(specs, keys, dkeys)):
        built = M.MPHF(outs[i])
        o = orc.build_mphf(k, leaf, 1000, bij, threads=THREADS, tree=tree)
        assert_same_function(o, built, k, dk)


def test_shockf2_l24_workload_in_full(torch, orc):
    w = W.WORKLOADS["shockf2_l24"]
    keys = W.keys_for(w)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, w.leaf, w.bucket, w.rotation, tree=w.tree)
    o = orc.build_mphf(keys, w.leaf, w.bucket, w.rotation, threads=THREADS, tree=w.tree)
    assert_same_function(o, g, keys, dkeys, full=False)
    assert g.info.gr_bits / w.n < 1.75  # about 1.67 bits per key (Appendix C's Pareto range)
