"""The launch-shape autotuner: every candidate shape builds the same function,
the fastest is cached per device, and tuned builds use it with unchanged output."""
import json

import numpy as np
import pytest

from paper_2212_09562_b300 import autotune as A
from paper_2212_09562_b300 import mphf as M
from paper_2212_09562_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_tune_caches_a_shape_and_tuned_builds_are_identical(tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("MPHF_TUNE_CACHE", str(tmp_path / "tune.json"))
    assert A.tuned(12, True) == A.DEFAULT
    rec = A.tune(12, True, n=200_000, bucket=1000, warm_s=0.5)
    assert (rec["threads"], rec["blocks_per_sm"], rec["seeds_per_thread"]) in A.CANDIDATES
    assert len(rec["candidates"]) == len(A.CANDIDATES)
    data = json.load(open(tmp_path / "tune.json"))
    assert len(data) == 1
    assert A.tuned(12, True) == (rec["threads"], rec["blocks_per_sm"], rec["seeds_per_thread"])
    keys = torch.from_numpy(W.distinct_u64(50_000, 77).view(np.int64)).cuda()
    a = M.MPHF.build(keys, 12, 1000, True, tuned=True).host_arrays()
    b = M.MPHF.build(keys, 12, 1000, True).host_arrays()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("spt", [1, 2, 4])
def test_seeds_per_thread_does_not_change_the_result(spt):
    """Every seeds-per-thread variant of the full lower-level split search
    stores the same values (l = 8, 12, 16; the oracle-checked default is the
    reference), alone and in a batch."""
    import torch
    for leaf, bucket, n in ((8, 100, 30_000), (12, 1000, 60_000), (16, 2000, 40_000)):
        keys = torch.from_numpy(W.distinct_u64(n, 7100 + leaf).view(np.int64)).cuda()
        a = M.MPHF.build(keys, leaf, bucket, True).host_arrays()
        b = M.MPHF.build(keys, leaf, bucket, True, seeds_per_thread=spt).host_arrays()
        for k in a:
            assert np.array_equal(a[k], b[k]), (leaf, spt, k)
    with pytest.raises(M.MPHFError):
        M.MPHF.build(keys, 16, 2000, True, seeds_per_thread=3)
