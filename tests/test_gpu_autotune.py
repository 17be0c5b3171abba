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
    rec = A.tune(12, True, n=200_000, bucket=1000)
    assert (rec["threads"], rec["blocks_per_sm"]) in A.CANDIDATES
    assert len(rec["candidates"]) == len(A.CANDIDATES)
    data = json.load(open(tmp_path / "tune.json"))
    assert len(data) == 1
    assert A.tuned(12, True) == (rec["threads"], rec["blocks_per_sm"])
    keys = torch.from_numpy(W.distinct_u64(50_000, 77).view(np.int64)).cuda()
    a = M.MPHF.build(keys, 12, 1000, True, tuned=True).host_arrays()
    b = M.MPHF.build(keys, 12, 1000, True).host_arrays()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
