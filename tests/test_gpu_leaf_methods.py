"""Leaf-search methods: lock-step brute force, early rejection at the first
collision, and early rejection with the rotation lookup table (Section 4,
"Lookup Tables") all store the same smallest value at every leaf, so each
must reproduce the oracle's function bit for bit."""
import numpy as np
import pytest

from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W
from test_gpu_parity import THREADS, assert_same_function, to_dev

pytestmark = pytest.mark.gpu

CASES = [(8, 100, False, 8, 5000), (8, 100, True, 16, 5000), (12, 1000, True, 8, 6000),
         (16, 2000, True, 8, 2500), (5, 7, True, 8, 3000), (16, 300, True, 8, 3001),
         (3, 40, False, 8, 800), (20, 3, True, 8, 700), (16, 17, False, 8, 400),
         (2, 5, True, 8, 500), (10, 250, False, 16, 2600)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_09562_b300 import build
    build.build()
    M.lib()
    return t


@pytest.mark.parametrize("method", [M.LEAF_LOCKSTEP, M.LEAF_EARLY, M.LEAF_TABLE])
@pytest.mark.parametrize("leaf,bucket,rotation,kb,n", CASES)
def test_leaf_methods_match_the_oracle(torch, orc, method, leaf, bucket, rotation, kb, n):
    keys = W.random_keys(n, kb, 3000 + 11 * n + leaf)
    o = orc.build_mphf(keys, leaf, bucket, rotation, threads=THREADS)
    dkeys = to_dev(torch, keys)
    g = M.MPHF.build(dkeys, leaf, bucket, rotation, leaf_method=method)
    assert_same_function(o, g, keys, dkeys)


@pytest.mark.parametrize("method", [M.LEAF_EARLY, M.LEAF_TABLE])
def test_leaf_methods_on_the_rot_l12_workload(torch, method):
    w = W.WORKLOADS["rot_l12"]
    keys = W.keys_for(w)
    dkeys = to_dev(torch, keys)
    a = M.MPHF.build(dkeys, w.leaf, w.bucket, w.rotation, leaf_method=M.LEAF_LOCKSTEP).host_arrays()
    b = M.MPHF.build(dkeys, w.leaf, w.bucket, w.rotation, leaf_method=method).host_arrays()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_bad_leaf_method_is_refused(torch):
    dkeys = to_dev(torch, W.distinct_u64(100, 1))
    with pytest.raises(M.MPHFError) as e:
        M.MPHF.build(dkeys, 8, 100, True, leaf_method=3)
    assert e.value.code == M.EINVAL


@pytest.mark.parametrize("method", [M.LEAF_EARLY, M.LEAF_TABLE])
def test_shockhash_leaves_ignore_the_leaf_method(torch, method):
    """ShockHash leaves have one search; the method of plain and rotation
    leaves does not change them."""
    dkeys = to_dev(torch, W.distinct_u64(30000, 5300))
    a = M.MPHF.build(dkeys, 16, 2000, M.SHOCKHASH).host_arrays()
    b = M.MPHF.build(dkeys, 16, 2000, M.SHOCKHASH, leaf_method=method).host_arrays()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
