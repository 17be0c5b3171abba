"""Builds from several host threads at once, each on its own stream.

The library keeps per-device tables behind locks and everything else per
call, so concurrent calls (ctypes releases the GIL during each) must give
the functions that one-at-a-time calls give.
"""
import threading

import numpy as np
import pytest

from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W
from test_gpu_parity import to_dev

pytestmark = pytest.mark.gpu

SPECS = [(8, 100, M.PLAIN, M.TREE_RECSPLIT), (12, 1000, M.ROTATION, M.TREE_RECSPLIT),
         (24, 2000, M.SHOCKHASH, M.TREE_FANOUT2), (10, 300, M.ROTATION, M.TREE_FANOUT2),
         (16, 500, M.SHOCKHASH, M.TREE_RECSPLIT), (5, 50, M.ROTATION, M.TREE_RECSPLIT)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2212_09562_b300 import build
    build.build()
    M.lib()
    return t


def test_concurrent_builds_equal_sequential_builds(torch):
    keys = [to_dev(torch, W.random_keys(30_000 + 1000 * i, 8, 900 + i)) for i in range(len(SPECS))]
    torch.cuda.synchronize()
    results, errors = [None] * len(SPECS), []

    def work(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                leaf, bucket, bij, tree = SPECS[i]
                g = M.MPHF.build(keys[i], leaf, bucket, bij, tree=tree, stream=s)
                results[i] = (g.host_arrays(), g.verify(keys[i], stream=s))
                g.close()
        except Exception as e:  # reported below
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(SPECS))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i, (leaf, bucket, bij, tree) in enumerate(SPECS):
        g = M.MPHF.build(keys[i], leaf, bucket, bij, tree=tree)
        arrays, bad = results[i]
        assert bad == 0
        for k, v in g.host_arrays().items():
            assert np.array_equal(arrays[k], v), (i, k)
